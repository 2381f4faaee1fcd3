// Render kernels of the f32 layout, fwd passes (the instantiations are spread over files so that they
// compile in parallel; fewer, larger files keep the library small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, false, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, false, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_TRACE, false, 0)
