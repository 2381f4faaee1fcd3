// Render kernels: f32 layout, bwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD, false, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD_STORE, false, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, false, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, false, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_NRM, false, false)
