// FP32-compensated instantiations of the particle pass: the other passes
// with their flags compiled in (second of three translation units).
#include "m2m_kernels.cuh"

namespace m2m {

// The step that also takes the (E, L_z) range, the first step after a
// prior recompute (no pending update, with or without the range) and the
// prior-cell pass, for the layout / potential pairs of the workloads (layout
// 0, the run-time set walk, with one logarithmic or Hernquist potential).
template <int FL, int L, int PK>
static void *one() { return (void *)k_pass<float, 1024, 1, L, 0, FL, PK>; }

template <int FL>
static void *other_pk(int layout, int pk) {
    if (layout == 0 && pk == PK_LOG) return one<FL, 0, PK_LOG>();
    if (layout == 0 && pk == PK_HERNQUIST) return one<FL, 0, PK_HERNQUIST>();
    if (layout == 1 && pk == PK_LOG) return one<FL, 1, PK_LOG>();
    if (layout == 2 && pk == PK_HERNQUIST) return one<FL, 2, PK_HERNQUIST>();
    if (layout == 2 && pk == PK_SH) return one<FL, 2, PK_SH>();
    if (layout == 2 && pk == PK_SH_TRI) return one<FL, 2, PK_SH_TRI>();
    if (layout == 2 && pk == PK_SH_FULL) return one<FL, 2, PK_SH_FULL>();
    if (layout == 2 && pk == PK_HERNQUIST_NFW) return one<FL, 2, PK_HERNQUIST_NFW>();
    if (layout == 3 && pk == PK_HERNQUIST) return one<FL, 3, PK_HERNQUIST>();
    if (layout == 4 && pk == PK_LOG) return one<FL, 4, PK_LOG>();
    return nullptr;
}

void *pass_kernel_f32_compiled(int flags, int layout, int pk) {
    switch (flags) {
        case F_STEADY: return pass_kernel_f32_steady(layout, pk);
        case F_STEADY | F_MINMAX: return other_pk<F_STEADY | F_MINMAX>(layout, pk);
        case F_PUSH | F_SCAT | F_STATS: return other_pk<F_PUSH | F_SCAT | F_STATS>(layout, pk);
        case F_PUSH | F_SCAT | F_STATS | F_MINMAX: return other_pk<F_PUSH | F_SCAT | F_STATS | F_MINMAX>(layout, pk);
        case F_CELLS | F_UPD: return other_pk<F_CELLS | F_UPD>(layout, pk);
        default: return nullptr;
    }
}

}  // namespace m2m
