// Instantiations of the persistent multi-step kernel (FP32C): the compiled
// observable layouts with the potential signatures of the workloads.
#include "m2m_steps.cuh"

namespace m2m {

void *steps_kernel_f32(int layout, int pk) {
    if (layout == 1 && pk == PK_LOG) return (void *)k_steps<1, PK_LOG>;
    if (layout == 2 && pk == PK_HERNQUIST) return (void *)k_steps<2, PK_HERNQUIST>;
    if (layout == 2 && pk == PK_HERNQUIST_NFW) return (void *)k_steps<2, PK_HERNQUIST_NFW>;
    if (layout == 3 && pk == PK_HERNQUIST) return (void *)k_steps<3, PK_HERNQUIST>;
    if (layout == 4 && pk == PK_LOG) return (void *)k_steps<4, PK_LOG>;
    return nullptr;
}

}  // namespace m2m
