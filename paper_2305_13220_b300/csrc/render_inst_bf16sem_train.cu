// Render kernels of the bf16sem layout, train passes (the instantiations are spread over files so that they
// compile in parallel; fewer, larger files keep the library small).
#include "render_kernels.cuh"

SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN, true, true)
SDG_INSTANTIATE_LAUNCH(sdg::PASS_TRAIN_BETA, true, true)
