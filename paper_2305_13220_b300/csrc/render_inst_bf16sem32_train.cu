// Render kernels of the bf16sem layout with 24-32 semantic channels, train passes (the
// instantiations are spread over files so that they compile in parallel; fewer, larger files keep the library
// small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, true, 32)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, true, 32)
