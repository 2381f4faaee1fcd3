// Render kernels of the bf16 layout, fwd passes (the instantiations are spread over files so that they
// compile in parallel; fewer, larger files keep the library small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, true, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, true, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_TRACE, true, 0)
