// Render kernels: bf16 layout, bwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD, true, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD_STORE, true, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, true, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, true, false)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_NRM, true, false)
