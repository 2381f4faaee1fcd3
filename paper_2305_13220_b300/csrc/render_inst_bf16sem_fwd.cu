// Render kernels: bf16sem layout, fwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, true, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, true, true)
