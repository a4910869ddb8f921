// pty_n128.cu -- the hot path instantiated for a 128 x 128 probe window.
#include "pipeline.cuh"

namespace pty {
template int run_pipeline<128>(const Problem& pb);
}  // namespace pty
