// Render kernels of the bf16sem layout with up to 20 semantic channels, fwd passes (the
// instantiations are spread over files so that they compile in parallel; fewer, larger files keep the library
// small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD, true, sdg::kSemCapSmall)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_STORE, true, sdg::kSemCapSmall)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_FWD_TRACE, true, sdg::kSemCapSmall)
