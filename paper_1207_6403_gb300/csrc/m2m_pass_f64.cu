// FP64 instantiations of the particle pass.
#include "m2m_kernels.cuh"

namespace m2m {

template <int NT, int MINB>
static void *pick_layout_f64(int layout) {
    switch (layout) {
        case 1: return (void *)k_pass<double, NT, MINB, 1, 0>;
        case 2: return (void *)k_pass<double, NT, MINB, 2, 0>;
        case 3: return (void *)k_pass<double, NT, MINB, 3, 0>;
        default: return (void *)k_pass<double, NT, MINB, 0, 0>;
    }
}

void *pass_kernel_f64(int threads, int layout) {
    switch (threads) {
        case 512: return pick_layout_f64<512, 1>(layout);
        default: return pick_layout_f64<256, 1>(layout);
    }
}

void *cells_kernel_f64() { return (void *)k_cells<double>; }

}  // namespace m2m
