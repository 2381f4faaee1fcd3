// Render kernels: f32 layout, fwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, false, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, false, false)
