// pty_n64.cu -- the hot path instantiated for a 64 x 64 probe window.
#include "pipeline.cuh"

namespace pty {
template int run_pipeline<64>(const Problem& pb);
}  // namespace pty
