// pty_n128.cu -- the hot path instantiated for a 128 x 128 probe window: the FP32 shared-memory FFT pass
// and the split-precision DFT-GEMM passes.  Both live in one translation unit so that the kernel
// templates they share are compiled (and given their launch attributes) once.
#include "dftgemm.cuh"

namespace pty {
template int run_pipeline<128>(const Problem& pb);
template int run_pipeline_gemm<128, PTY_FFT_SPLIT_BF16>(const Problem& pb);
template int run_pipeline_gemm<128, PTY_FFT_SPLIT_FP16>(const Problem& pb);
template int run_pipeline_gemm<128, PTY_FFT_SPLIT3_BF16>(const Problem& pb);
}  // namespace pty
