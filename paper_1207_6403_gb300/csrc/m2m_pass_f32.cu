// FP32-compensated instantiations of the particle pass: the run-time-flag
// kernels and the steady-state step (one of three translation units for
// FP32C, so that the library builds in parallel).
#include "m2m_kernels.cuh"

namespace m2m {

template <int NT, int MINB>
static void *pick_layout_f32(int layout) {
    switch (layout) {
        case 1: return (void *)k_pass<float, NT, MINB, 1, 0>;
        case 2: return (void *)k_pass<float, NT, MINB, 2, 0>;
        case 3: return (void *)k_pass<float, NT, MINB, 3, 0>;
        case 4: return (void *)k_pass<float, NT, MINB, 4, 0>;
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

// The steady-state step (pending update + push + scatter + stats) with its
// flags compiled in (1024 threads, plain loads), for every layout (0: the
// run-time set walk) and potential signature (PK_ANY: the run-time
// component walk).
template <int L>
static void *steady_pk(int pk) {
    switch (pk) {
        case PK_HERNQUIST: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_HERNQUIST>;
        case PK_LOG: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_LOG>;
        case PK_SH: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_SH>;
        case PK_SH_TRI:     // the triaxial expansion: the layout of its workload (shells + annuli)
            if constexpr (L == 2) return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_SH_TRI>;
            return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY>;
        case PK_SH_FULL:    // the full expansion (l <= 4): the same layout
            if constexpr (L == 2) return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_SH_FULL>;
            return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY>;
        case PK_HERNQUIST_NFW: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY, PK_HERNQUIST_NFW>;
        default: return (void *)k_pass<float, 1024, 1, L, 0, F_STEADY>;
    }
}

void *pass_kernel_f32_steady(int layout, int pk) {
    switch (layout) {
        case 0: return steady_pk<0>(pk);
        case 1: return steady_pk<1>(pk);
        case 2: return steady_pk<2>(pk);
        case 3: return steady_pk<3>(pk);
        case 4:     // lookup-table apertures: the logarithmic potential of their workload
            return pk == PK_LOG ? (void *)k_pass<float, 1024, 1, 4, 0, F_STEADY, PK_LOG>
                                : (void *)k_pass<float, 1024, 1, 4, 0, F_STEADY>;
        default: return nullptr;
    }
}

void *cells_kernel_f32() { return (void *)k_cells<float>; }

}  // namespace m2m
