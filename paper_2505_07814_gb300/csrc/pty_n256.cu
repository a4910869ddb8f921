// pty_n256.cu -- the hot path instantiated for a 256 x 256 probe window (four-CTA clusters).
#include "pipeline.cuh"

namespace pty {
template int run_pipeline<256>(const Problem& pb);
}  // namespace pty
