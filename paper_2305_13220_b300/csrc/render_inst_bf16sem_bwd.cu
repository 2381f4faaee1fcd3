// Render kernels: bf16sem layout, bwd pass instantiations.
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD, true, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_BWD_STORE, true, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, true, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, true, true)
