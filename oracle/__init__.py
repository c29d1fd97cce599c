"""Plain FP64 CPU oracle for rBKI-TK and rBKI-TK-TR.  TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import or run anything in this package.  The product path (the CUDA library and
its Python binding) never calls it, and this package never imports the product
package: the two share no code.  The only common dependency is the seeded input
generator module `synth`, which holds no arithmetic of the method.

Every function follows a passage of the paper (arXiv 2211.14828) and cites it:
  * philox.py   - the sketching matrix Omega: Philox4x32-10 (Salmon et al., SC'11)
                  + Box-Muller, an explicit counter-based definition of the
                  "randomized sketching matrix" of Algorithm 1, step 1.
  * tensor.py   - mode-n unfolding, mode-n product, Tucker / TR models
                  (Sec. 2.1, Eqs. TKD, unTKD, TR).
  * rbki.py     - rBKI tensor sketching (Algorithm 1), rBKI-TK (Algorithm 2),
                  Remark 1 (Z = Q^T X X^T Q), Eq. tensorsketch, truncated HOSVD.
  * tr.py       - TR-ALS on the Tucker core and rBKI-TK-TR (Algorithm 3).
  * metrics.py  - Fit, RErr, PSNR (Sec. 4 metrics) and Eq. SNR.

Parity status per function is stated in each module header; functions without a
pin independent of themselves say "parity unpinned".
"""
from . import philox, tensor, rbki, tr, metrics  # noqa: F401
