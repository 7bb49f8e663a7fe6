// FP32-compensated instantiations of the particle pass: the bulk-copy
// pipeline and the batched passes (third of three translation units).
#include "m2m_kernels.cuh"

namespace m2m {

// The compiled layouts with the block-level bulk-copy pipeline (1024 threads).
void *pass_kernel_f32_pipe(int layout) {
    switch (layout) {
        case 1: return (void *)k_pass<float, 1024, 1, 1, 1>;
        case 2: return (void *)k_pass<float, 1024, 1, 2, 1>;
        case 3: return (void *)k_pass<float, 1024, 1, 3, 1>;
        default: return nullptr;
    }
}

void *pass_kernel_f32_pipe_steady(int layout) {
    switch (layout) {
        case 1: return (void *)k_pass<float, 1024, 1, 1, 1, F_STEADY>;
        case 2: return (void *)k_pass<float, 1024, 1, 2, 1, F_STEADY>;
        case 3: return (void *)k_pass<float, 1024, 1, 3, 1, F_STEADY>;
        default: return nullptr;
    }
}

// All models of a batch in one launch (compiled layouts, plain loads); the
// steady-state step with its flags compiled in.
void *pass_kernel_f32_batch(int layout, bool steady, int pk) {
    if (steady) {
        // the batched trial-potential models: Hernquist stars in Hernquist + NFW
        if (layout == 2 && pk == PK_HERNQUIST_NFW) return (void *)k_pass_batch<float, 1024, 1, 2, F_STEADY, PK_HERNQUIST_NFW>;
        switch (layout) {
            case 1: return (void *)k_pass_batch<float, 1024, 1, 1, F_STEADY>;
            case 2: return (void *)k_pass_batch<float, 1024, 1, 2, F_STEADY>;
            case 3: return (void *)k_pass_batch<float, 1024, 1, 3, F_STEADY>;
            case 4: return (void *)k_pass_batch<float, 1024, 1, 4, F_STEADY>;
            default: break;
        }
    }
    switch (layout) {
        case 1: return (void *)k_pass_batch<float, 1024, 1, 1>;
        case 2: return (void *)k_pass_batch<float, 1024, 1, 2>;
        case 3: return (void *)k_pass_batch<float, 1024, 1, 3>;
        case 4: return (void *)k_pass_batch<float, 1024, 1, 4>;
        default: return (void *)k_pass_batch<float, 1024, 1, 0>;
    }
}

}  // namespace m2m
