// Render kernels of the bf16sem layout with 24-32 semantic channels, fwd passes (the
// instantiations are spread over files so that they compile in parallel; fewer, larger files keep the library
// small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, true, 32)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, true, 32)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_TRACE, true, 32)
