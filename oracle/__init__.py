"""CPU oracle for the selective-encryption hot path (first level of protection, Sect. 6.3.1).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the build entry point and
the CPU-baseline leg of the benchmark may import this package.  The product (the CUDA
library and its Python binding) never calls it, and it shares no code, table or constant
generator with the CUDA path.

Plain, slow, obviously correct code, following the paper step by step:

  dct.py    8x8 DCT-II per channel in float64 (Sect. 6.4.2: separable 1-D basis)
  exact.py  exact arithmetic in Z[cos(pi/16)] used to take every rounding decision on
            the exact real value (Sect. 6.4.3: "numbers are turned back to integer")
  aes.py    AES-128 written from FIPS-197 (S-box generated from its definition) and the
            CTR mode of NIST SP 800-38A (Sect. 6.12: "AES with counter mode")
  fds.py    protect / restore: DCT -> int16 -> zigzag split -> AES-CTR on Part 1, and the
            inverse (Sect. 6.3.1, Fig. 6; Sect. 3.2 defragmentation)
  pack.py   11-bit and 8-bit packed storage of the fragments (Sect. 6.4.3, Table 5)
  public.py the public fragment as an image (Sect. 6.5.1, Fig. 10) and the histogram /
            adjacent-pixel correlation statistics (Sect. 6.6)
  strong.py strong level: public image XOR SHA-512 of Part 1 per block (Sect. 6.3.2, Fig. 8)
  dwt.py    the lossless DWT scheme: Le Gall 5/3 lifting, AES-CTR on level 1, SHA-256 /
            SHA-512 masks on levels 2 and 3 (Sect. 6.8-6.12, Fig. 18)

Every function that is not pinned by a test against something other than itself says
"parity unpinned" in its docstring.  None does at present.
"""
from . import aes, dct, dwt, exact, fds, pack, public, strong  # noqa: F401
