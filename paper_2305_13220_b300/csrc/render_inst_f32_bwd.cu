// Render kernels of the f32 layout, bwd passes (the instantiations are spread over files so that they
// compile in parallel; fewer, larger files keep the library small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD, false, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD_STORE, false, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, false, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, false, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_NRM, false, 0)
