// Analysis kernels outside the step: the velocity-ellipsoid moments of the
// anisotropy analysis and the gather of a batch's records.
#pragma once
#include "m2m_kernels.cuh"

namespace m2m {

// Velocity-ellipsoid moments per spherical shell: block-private double sums
// in shared memory (4 per shell), then one global atomic per sum.  The
// shell is the last edge <= r^2 (r^2 in the state precision, compared in
// double), by bisection over the edges in shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_vmoments(const R *x, const R *y, const R *z, const R *vx, const R *vy,
                                                  const R *vz, const double *w, long long n, const double *e2,
                                                  int nsh, double *out) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *acc = (double *)smem;
    double *ed = acc + 4 * nsh;
    for (int k = threadIdx.x; k < 4 * nsh; k += blockDim.x) acc[k] = 0.0;
    for (int k = threadIdx.x; k <= nsh; k += blockDim.x) ed[k] = e2[k];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const R xs = x[i], ys = y[i], zs = z[i];
        const double r2 = (double)((xs * xs + ys * ys) + zs * zs);
        if (!(r2 >= ed[0] && r2 < ed[nsh])) continue;      // outside (or NaN)
        int lo = 0, hi = nsh;                               // ed[lo] <= r2 < ed[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ed[mid] <= r2) lo = mid; else hi = mid;
        }
        const double X = xs, Y = ys, Z = zs, U = vx[i], V = vy[i], W = vz[i];
        const double r = sqrt(X * X + Y * Y + Z * Z), Rc = sqrt(X * X + Y * Y);
        const double vr = r > 0 ? (X * U + Y * V + Z * W) / r : 0.0;
        const double vp = Rc > 0 ? (X * V - Y * U) / Rc : 0.0;
        const double v2 = U * U + V * V + W * W;
        const double wi = w[i];
        atomicAdd(acc + 4 * lo, wi);
        atomicAdd(acc + 4 * lo + 1, wi * (vr * vr));
        atomicAdd(acc + 4 * lo + 2, wi * ((v2 - vr * vr) - vp * vp));
        atomicAdd(acc + 4 * lo + 3, wi * (vp * vp));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 4 * nsh; k += blockDim.x)
        if (acc[k] != 0.0) atomicAdd(out + k, acc[k]);
}

// The last record and the error word of every model of a batch into one
// array each (one thread per model).
__global__ void k_gather_records(const m2m_record *const *src, const int *const *err, int n, m2m_record *dst,
                                 int *err_out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) {
        dst[m] = *src[m];
        err_out[m] = *err[m];
    }
}

// ----------------------------------------------------- particle shards
// A shard's exchange buffers after its scatter pass (one warp): the int64
// observable totals copied out (and cleared for the next scatter), the
// entropy and weight partials of the pass's blocks summed in block order,
// and, when the pass took the (E, L_z) range, the block ranges reduced to
// (min E, -max E, -max |L_z|) so that a single minimum over shards gives
// the global range.
template <class R>
__global__ void k_shard_pack(unsigned long long *y_acc, long long *totals, int nobs, const double *stat_slots,
                             int nblk, double *stats, const void *mm_slots, int mm_nblk, double *range) {
    for (int j = threadIdx.x; j < nobs; j += blockDim.x) {
        totals[j] = (long long)y_acc[j];
        y_acc[j] = 0ull;
    }
    if (threadIdx.x == 0) {
        double s = 0.0, w = 0.0;
        for (int b = 0; b < nblk; ++b) { s += stat_slots[2 * b]; w += stat_slots[2 * b + 1]; }
        stats[0] = s;
        stats[1] = w;
        if (range && mm_nblk > 0) {
            const R *mm = (const R *)mm_slots;
            double e0 = (double)mm[0], e1 = (double)mm[1], l = (double)mm[2];
            for (int b = 1; b < mm_nblk; ++b) {
                e0 = fmin(e0, (double)mm[4 * b]);
                e1 = fmax(e1, (double)mm[4 * b + 1]);
                l = fmax(l, (double)mm[4 * b + 2]);
            }
            range[0] = e0;
            range[1] = -e1;
            range[2] = -l;
        }
    }
}

// The global range back into the range slots the prior-cell pass reads
// (one slot), in the state precision (each value is one the shards' passes
// produced, so the conversion is exact).
template <class R>
__global__ void k_shard_range(const double *range, void *mm_slots) {
    R *mm = (R *)mm_slots;
    mm[0] = (R)range[0];
    mm[1] = (R)(-range[1]);
    mm[2] = (R)(-range[2]);
    mm[3] = R(0);
}

// Philox4x32-10 output words of given counters and keys, one thread per
// draw: the generator of the seeing draws, exposed for its known-answer
// check.
__global__ void k_philox_words(const unsigned *ctr, const unsigned *key, long long n, unsigned *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 o = philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]),
                                  make_uint2(key[2 * i], key[2 * i + 1]));
    out[4 * i] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
}

}  // namespace m2m
