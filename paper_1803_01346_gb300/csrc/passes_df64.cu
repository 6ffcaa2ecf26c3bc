// passes_df64.cu - the shared-memory FFT passes instantiated for the double-float element type
// (SCFFT_PREC_DF64); a translation unit of its own so that it compiles beside passes.cu.
#include "passes_impl.cuh"

namespace scfft {

INST_PASSES(dfloat)

}  // namespace scfft
