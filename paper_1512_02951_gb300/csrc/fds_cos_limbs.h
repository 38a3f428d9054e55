/* Generated by gen_cos_limbs.py: floor(cos(j pi/16) * 2^256), j = 1..7, as eight
 * 32-bit limbs, least significant first (an initializer for uint32_t[7][8]). */
#pragma once
#define FDS_COS_LIMBS_INIT \
  { \
    {0xb48e8b1bu, 0xb1997321u, 0xd8f18ae1u, 0xc5f40e3fu, 0xfd2a722eu, 0x2172a361u, 0xbae58156u, 0xfb14be7fu}, /* j = 1 */ \
    {0x84083746u, 0xdb897c23u, 0xd0dae9b5u, 0xf0a83d3cu, 0xac1d6180u, 0x7e610231u, 0x946a3145u, 0xec835e79u}, /* j = 2 */ \
    {0x7cd39544u, 0xac08e58au, 0x99ec9eaau, 0xb4691d2fu, 0xdac83e68u, 0xf630e8b6u, 0x750d1819u, 0xd4db3148u}, /* j = 3 */ \
    {0x83339915u, 0xed17ac85u, 0x893ba84cu, 0x1d6f60bau, 0x754abe9fu, 0x597d89b3u, 0xf9de6484u, 0xb504f333u}, /* j = 4 */ \
    {0xc296fd79u, 0xca996068u, 0xadfba33eu, 0x7ca7d749u, 0xbff54867u, 0xbba4cfecu, 0x73464364u, 0x8e39d9cdu}, /* j = 5 */ \
    {0x62718f71u, 0x3a3c1590u, 0xab3de24cu, 0xbdf1f5b4u, 0xcf7eee1bu, 0x98916152u, 0xbaa58b46u, 0x61f78a9au}, /* j = 6 */ \
    {0x895414c1u, 0x39438767u, 0x12972f1du, 0xf394e58du, 0x93f33613u, 0x97323003u, 0xd34c156cu, 0x31f17078u}, /* j = 7 */ \
  }
/* round(cos(j pi/16) * 2^62), j = 1..7 */
#define FDS_COS_Q62_INIT \
  {4523073764714963030ll, 4260642322793532497ll, 3834476785802888710ll, 3260954456333195553ll, 2562115475870945497ll, 1764815834521887442ll, 899695310372275547ll}
