// Render kernels: f32sem layout, bwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD, false, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD_STORE, false, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, false, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, false, true)
