"""Plain, slow FP64 CPU oracle for the FFT-based 3D bulk-magnetization method
(Prigozhin & Sokolovsky, "3D simulation of superconducting magnetic shields and
lenses using the FFT", §2, Eqs. 1-7).

This package is TEST INFRASTRUCTURE. Only the test suite, the smoke check of the
package entry point and the CPU-baseline leg of the benchmark may import it.
The product path (the CUDA library and its Python binding) never imports or
calls it, and it shares no code with that path.
"""

from .scfft_oracle import *  # noqa: F401,F403
