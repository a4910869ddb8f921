// pty_n64.cu -- the hot path instantiated for a 64 x 64 probe window: the FP32 shared-memory FFT pass
// and the split-precision DFT-GEMM passes.  Both live in one translation unit so that the kernel
// templates they share are compiled (and given their launch attributes) once.
#include "dftgemm.cuh"

namespace pty {
template int run_pipeline<64>(const Problem& pb);
template int run_pipeline_gemm<64, PTY_FFT_SPLIT_BF16>(const Problem& pb);
template int run_pipeline_gemm<64, PTY_FFT_SPLIT_FP16>(const Problem& pb);
template int run_pipeline_gemm<64, PTY_FFT_SPLIT3_BF16>(const Problem& pb);
}  // namespace pty
