// Render kernels: f32sem layout, fwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, false, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, false, true)
