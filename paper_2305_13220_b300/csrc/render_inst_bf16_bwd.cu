// Render kernels of the bf16 layout, bwd passes (the instantiations are spread over files so that they
// compile in parallel; fewer, larger files keep the library small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD, true, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD_STORE, true, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, true, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, true, 0)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_NRM, true, 0)
