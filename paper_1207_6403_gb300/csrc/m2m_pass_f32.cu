// FP32-compensated instantiations of the particle pass (one translation
// unit per precision so the library builds in parallel).
#include "m2m_kernels.cuh"

namespace m2m {

template <int NT, int MINB>
static void *pick_layout_f32(int layout) {
    switch (layout) {
        case 1: return (void *)k_pass<float, NT, MINB, 1, 0>;
        case 2: return (void *)k_pass<float, NT, MINB, 2, 0>;
        case 3: return (void *)k_pass<float, NT, MINB, 3, 0>;
        default: return (void *)k_pass<float, NT, MINB, 0, 0>;
    }
}

void *pass_kernel_f32(int threads, int layout) {
    switch (threads) {
        case 256: return pick_layout_f32<256, 2>(layout);
        case 1024: return pick_layout_f32<1024, 1>(layout);
        default: return pick_layout_f32<512, 2>(layout);
    }
}

// The compiled layouts with the block-level bulk-copy pipeline (1024 threads).
void *pass_kernel_f32_pipe(int layout) {
    switch (layout) {
        case 1: return (void *)k_pass<float, 1024, 1, 1, 1>;
        case 2: return (void *)k_pass<float, 1024, 1, 2, 1>;
        case 3: return (void *)k_pass<float, 1024, 1, 3, 1>;
        default: return nullptr;
    }
}

// The steady-state step (pending update + push + scatter + stats) with its
// flags compiled in (1024 threads, plain loads), for each compiled layout
// and potential signature (PK_ANY: the run-time component walk).
template <int L>
static void *steady_pk(int pk) {
    switch (pk) {
        case PK_HERNQUIST: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_HERNQUIST>;
        case PK_LOG: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_LOG>;
        case PK_SH: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_SH>;
        case PK_HERNQUIST_NFW: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_HERNQUIST_NFW>;
        default: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY>;
    }
}
void *pass_kernel_f32_steady(int layout, int pk) {
    switch (layout) {
        case 1: return steady_pk<1>(pk);
        case 2: return steady_pk<2>(pk);
        case 3: return steady_pk<3>(pk);
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
            default: break;
        }
    }
    switch (layout) {
        case 1: return (void *)k_pass_batch<float, 1024, 1, 1>;
        case 2: return (void *)k_pass_batch<float, 1024, 1, 2>;
        case 3: return (void *)k_pass_batch<float, 1024, 1, 3>;
        default: return (void *)k_pass_batch<float, 1024, 1, 0>;
    }
}

void *cells_kernel_f32() { return (void *)k_cells<float>; }

}  // namespace m2m
