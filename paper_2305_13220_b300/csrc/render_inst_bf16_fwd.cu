// Render kernels: bf16 layout, fwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, true, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, true, false)
