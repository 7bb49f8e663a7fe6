// Kernels of the M2M step.
//
// k_pass      one streaming pass over the particles that does, per particle
//             and as the flags ask: the weight update pending from the last
//             residual (at the current positions), the entropy / total
//             weight partials, the KDK push, the weighted scatter into a
//             block-private shared histogram (flushed once per block into a
//             per-block slot), the (E, L_z) range for the priors, and the
//             prior-cell assignment with block-private cell sums.
// k_residual  per-bin reduction of the block slots in a fixed order, the
//             residuals, smoothing and coefficients, chi^2 by a warp-shuffle
//             reduction and, in the last block to finish, the step record.
// k_prior_mean, k_prior_gather
//             cell means sum/count and w_hat_i = mean of i's cell.
// k_cells     cell export for tests.
#pragma once
#include <limits.h>
#include <math.h>
#include <type_traits>
#include "m2m_device.cuh"
#include "m2m.h"

namespace m2m {

__device__ __forceinline__ float ceil_to(double e, float *) {
    float f = __double2float_rn(e);
    if ((double)f < e) f = nextafterf(f, INFINITY);
    return f;
}
__device__ __forceinline__ double ceil_to(double e, double *) { return e; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Knuth's two-sum: s + e == a + b exactly (round to nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (h, l) += (bh, bl) in float-float arithmetic (about 44 significant bits).
__device__ __forceinline__ void ff_add(float &h, float &l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    e = e + (l + bl);
    h = s + e;
    l = e - (h - s);
}

// Deterministic block sums of two per-thread float partials (FP32C entropy
// and weight partials) in float-float arithmetic: a fixed shuffle tree in
// each warp, the same over the warps' pairs in warp 0, then one conversion
// to double.  No FP64 work per thread or per warp: FP64 instructions issue
// at a small fraction of the FP32 rate on this part (even with one active
// lane), and a double tree over 1024 threads costs microseconds per block.
// red: 128 floats of shared memory; results valid in thread 0.
__device__ __forceinline__ void warp_ff2(float &ah, float &al, float &bh, float &bl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ph = __shfl_xor_sync(0xffffffffu, ah, o), pl = __shfl_xor_sync(0xffffffffu, al, o);
        const float qh = __shfl_xor_sync(0xffffffffu, bh, o), ql = __shfl_xor_sync(0xffffffffu, bl, o);
        ff_add(ah, al, ph, pl);
        ff_add(bh, bl, qh, ql);
    }
}
__device__ __forceinline__ void block_sum2_ff(float a, float b, float *red, double &ra, double &rb) {
    float ah = a, al = 0.f, bh = b, bl = 0.f;
    warp_ff2(ah, al, bh, bl);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    if (lane == 0) {
        red[wp] = ah; red[32 + wp] = al; red[64 + wp] = bh; red[96 + wp] = bl;
    }
    __syncthreads();
    if (wp == 0) {
        const bool in = lane < nw;
        ah = in ? red[lane] : 0.f; al = in ? red[32 + lane] : 0.f;
        bh = in ? red[64 + lane] : 0.f; bl = in ? red[96 + lane] : 0.f;
        warp_ff2(ah, al, bh, bl);
        if (lane == 0) {
            ra = (double)ah + (double)al;
            rb = (double)bh + (double)bl;
        }
    }
}

// Deterministic block sum (fixed shape), result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    return t;
}

// ----------------------------------------------------------------- priors
// Grid of the prior cells from the range slots of the preceding k_pass
// (F_MINMAX): interior edges lo + k*((hi-lo)/n) in double, held as the
// smallest R >= edge.  pe/pl are indexed 0..n (entries 1..n-1 used).
template <class R>
__device__ void prior_setup(const PassArgs &a, R *pe, R *pl, float *gp) {
    __shared__ double red[3][32];
    const R *mm = (const R *)a.mm_slots;
    R emin = R(INFINITY), emax = R(-INFINITY), lm = R(0);
    for (int b = threadIdx.x; b < a.mm_nblocks; b += blockDim.x) {
        emin = fmin(emin, mm[4 * b + 0]);
        emax = fmax(emax, mm[4 * b + 1]);
        lm = fmax(lm, mm[4 * b + 2]);
    }
    double de = (double)emin, dx = (double)emax, dl = (double)lm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        de = fmin(de, __shfl_xor_sync(0xffffffffu, de, o));
        dx = fmax(dx, __shfl_xor_sync(0xffffffffu, dx, o));
        dl = fmax(dl, __shfl_xor_sync(0xffffffffu, dl, o));
    }
    int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) { red[0][wp] = de; red[1][wp] = dx; red[2][wp] = dl; }
    __syncthreads();
    __shared__ double rng[4];
    if (threadIdx.x == 0) {
        double a0 = red[0][0], a1 = red[1][0], a2 = red[2][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            a0 = fmin(a0, red[0][k]); a1 = fmax(a1, red[1][k]); a2 = fmax(a2, red[2][k]);
        }
        // (E, L_z): [min E, max E] x [-max |L_z|, max |L_z|]; (E, L^2):
        // [min E, max E] x [0, max L^2]; (E, L/L_c): [min E, 0) x [0, 1]
        const bool lz = a.prior_kind == M2M_PRIOR_E_LZ, l2 = a.prior_kind == M2M_PRIOR_E_L2;
        double lo = a0, hi = (lz || l2) ? a1 : 0.0;
        double l0 = lz ? -a2 : 0.0;
        double l1 = (lz || l2) ? a2 : 1.0;
        rng[0] = lo; rng[1] = (hi - lo) / (double)a.nE;
        rng[2] = l0; rng[3] = (l1 - l0) / (double)a.nL;
    }
    __syncthreads();
    double lo = rng[0], we = rng[1], l0 = rng[2], wl = rng[3];
    for (int k = threadIdx.x; k <= a.nE; k += blockDim.x)
        pe[k] = (k >= 1 && k < a.nE) ? ceil_to(lo + (double)k * we, (R *)nullptr) : R(0);
    for (int k = threadIdx.x; k <= a.nL; k += blockDim.x)
        pl[k] = (k >= 1 && k < a.nL) ? ceil_to(l0 + (double)k * wl, (R *)nullptr) : R(0);
    if (threadIdx.x == 0) {
        gp[0] = we > 0 ? (float)(1.0 / we) : 0.f;
        gp[1] = we > 0 ? (float)(-lo / we) : 0.f;
        gp[2] = wl > 0 ? (float)(1.0 / wl) : 0.f;
        gp[3] = wl > 0 ? (float)(-l0 / wl) : 0.f;
    }
    __syncthreads();
}

// Order-preserving integer key of a float that is not NaN (-0 below +0)
// and its inverse.
__device__ __forceinline__ int fkey(float v) {
    const int b = __float_as_int(v);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float fkey_inv(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// E and the second integral of the prior: L_z, or L^2 = (Lx*Lx + Ly*Ly) +
// Lz*Lz for the (E, L^2) cells (its range is [0, max |L^2|] as the L_z
// range is [-max |L_z|, max |L_z|]).
template <class R, int PK = PK_ANY>
__device__ __forceinline__ void energy_lz(R x, R y, R z, R vx, R vy, R vz, const PassArgs &a, const R *sh,
                                          R &E, R &Lz) {
    R v2 = (vx * vx + vy * vy) + vz * vz;
    E = R(0.5) * v2 + potential<R, PK>(x, y, z, a, sh);
    Lz = x * vy - y * vx;
    if (a.prior_kind == M2M_PRIOR_E_L2) {
        const R Lx = y * vz - z * vy, Ly = z * vx - x * vz;
        Lz = (Lx * Lx + Ly * Ly) + Lz * Lz;
    }
}

template <class R, int PK = PK_ANY>
__device__ __forceinline__ int prior_cell(R x, R y, R z, R vx, R vy, R vz, const PassArgs &a,
                                          const R *pe, const R *pl, const float *gp, const R *sh) {
    R E, Lz;
    energy_lz<R, PK>(x, y, z, vx, vy, vz, a, sh, E, Lz);
    if (a.prior_kind == M2M_PRIOR_E_LZ || a.prior_kind == M2M_PRIOR_E_L2) {
        int iE = count_le<R>(E, pe, a.nE, gp[0], gp[1]);
        int iL = count_le<R>(Lz, pl, a.nL, gp[2], gp[3]);       // L_z or L^2
        return iE * a.nL + iL;
    }
    // E_LC: Hernquist circular-orbit angular momentum at energy E
    if (E >= R(0)) return a.nE * a.nL;
    R Lx = y * vz - z * vy;
    R Ly = z * vx - x * vz;
    R L2 = (Lx * Lx + Ly * Ly) + Lz * Lz;
    R ed = E * KC(R, a.pk, a.f_pk);
    R sq = sqrt(R(1) - R(8) * ed);
    R s = (R(-1) - sq) / (R(4) * ed);
    R sm = s - R(1);
    R Lc2 = KC(R, a.pgma, a.f_pgma) * (((sm * sm) * sm) / (s * s));
    R X = L2 / Lc2;
    int iE = count_le<R>(E, pe, a.nE, gp[0], gp[1]);
    int iL = count_le<R>(X, pl, a.nL, gp[2], gp[3]);
    return iE * a.nL + iL;
}

// ----------------------------------------------------------------- record
// The step record from the residual's per-block partials (chi^2, sum of
// Delta^2, max |Delta~|: 3 doubles per block) and the pass's per-block
// partials (S, sum w: 2 doubles per block), reduced by one warp in a fixed
// order (lane k takes blocks k, k+32, ... in turn, then a fixed shuffle
// tree): the same record whichever kernel computes it.  Lane 0 writes it.
__device__ __forceinline__ void record_warp(const double *chi, int nch, const double *st, int nst, double mu,
                                            long long step, int write_ring, m2m_record *ring, m2m_record *last,
                                            int *err) {
    const int lane = threadIdx.x & 31;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0;
    // up to 8 partials per lane loaded before any is added (one memory
    // latency instead of eight), then added in block order
    constexpr int U = 8;
    for (int b0 = lane; b0 < nch; b0 += 32 * U) {
        double t0[U], t1[U], t2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + 32 * u;
            const bool ok = b < nch;
            t0[u] = ok ? __ldcg(chi + 3 * b) : 0.0;
            t1[u] = ok ? __ldcg(chi + 3 * b + 1) : 0.0;
            t2[u] = ok ? __ldcg(chi + 3 * b + 2) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) { v0 += t0[u]; v1 += t1[u]; v2 = fmax(v2, t2[u]); }
    }
    for (int b0 = lane; b0 < nst; b0 += 32 * U) {
        double t3[U], t4[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + 32 * u;
            const bool ok = b < nst;
            t3[u] = ok ? __ldcg(st + 2 * b) : 0.0;
            t4[u] = ok ? __ldcg(st + 2 * b + 1) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) { v3 += t3[u]; v4 += t4[u]; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 = fmax(v2, __shfl_xor_sync(0xffffffffu, v2, o));
        v3 += __shfl_xor_sync(0xffffffffu, v3, o);
        v4 += __shfl_xor_sync(0xffffffffu, v4, o);
    }
    if (lane == 0) {
        m2m_record r;
        r.step = step;
        r.chi2 = v0; r.chi2_raw = v1; r.S = v3; r.sum_w = v4;
        r.F = -0.5 * v0 + mu * v3;
        r.max_abs_dt = v2;
        *last = r;
        if (write_ring) ring[step % M2M_HISTORY] = r;
        if (!(isfinite(v0) && isfinite(v3) && isfinite(v4))) atomicOr(err, ERR_NONFINITE);
    }
}

// ----------------------------------------------------------------- staging
// Copy n elements of T from global to shared memory, every load of a thread
// issued before its stores: 16-byte vectors (src and dst 16-byte aligned),
// up to U per thread in registers, then the scalar tail.  A plain loop that
// stores each element before loading the next waits one memory latency per
// element, since a store through a generic pointer may alias the next load.
// `src` may be written by the preceding kernel (read past L1).
template <int U, class T>
__device__ __forceinline__ void stage(T *dst, const T *src, int n, int tid, int nt) {
    constexpr int V = 16 / sizeof(T);
    const int n4 = n / V;
    const int4 *s4 = (const int4 *)src;
    int4 *d4 = (int4 *)dst;
    int4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int k = tid + u * nt;
        if (k < n4) v[u] = __ldcg(s4 + k);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int k = tid + u * nt;
        if (k < n4) d4[k] = v[u];
    }
    for (int k = tid + U * nt; k < n4; k += nt) d4[k] = __ldcg(s4 + k);
    for (int k = V * n4 + tid; k < n; k += nt) dst[k] = src[k];
}

// ----------------------------------------------------------------- k_pass
// Dynamic shared memory of pass_body (host side; the same order and
// rounding as the carve-up at the top of pass_body, without the pipeline's
// stage buffers).  sh_len: SH node-table values staged when the pass pushes.
inline size_t pass_smem_bytes(bool f32, int layout, int flags, int nobs, int edge_len, int gh_len, int sh_len,
                              int nE, int nL, int ncells, int pmap_len = 0) {
    const size_t rs = f32 ? 4 : 8;
    size_t b = 0;
    if (flags & F_SCAT) b += f32 ? 12 * (size_t)((nobs + 3) & ~3) : 8 * (size_t)((nobs + 1) & ~1);
    if (flags & F_UPD) b += rs * (size_t)((nobs + 3) & ~3);
    b += rs * (size_t)((edge_len + 3) & ~3);
    b += 2 * rs * (size_t)((edge_len + 1) & ~1);                     // edge pairs
    b += rs * (size_t)((gh_len + 3) & ~3);
    if (f32 && layout != 0) b += 48 * (size_t)(gh_len / 5);          // combined GH records
    else if (flags & F_UPD) b += rs * (size_t)((gh_len + 3) & ~3);
    if (f32 && layout == 1) b += 2 * (size_t)((pmap_len + 7) & ~7);   // pixel -> aperture table
    if (sh_len && (flags & (F_PUSH | F_MINMAX | F_CELLS))) b += rs * (size_t)((sh_len + 3) & ~3);
    if (flags & F_CELLS) {
        b += rs * (size_t)((nE + 4) & ~3) + rs * (size_t)((nL + 4) & ~3) + 16;
        if (f32) b += 12 * (size_t)((ncells + 3) & ~3);
        else b += 8 * (size_t)((ncells + 1) & ~1) + 4 * (size_t)((ncells + 3) & ~3);
    }
    return b;
}

template <class R>
struct PassSmem {
    int *hL, *hM, *hH;       // FP32C histogram: V = H * 2^32 + M * 2^16 + L per bin (exact fixed point)
    double *h_d;             // FP64 histogram
    const R *coef, *edges, *gh;
    const Pair<R> *epair;    // (e[k], e[k+1]) for every edge-table index k
    const R *gpoly;          // per GH cell: norm * sum_n coef_n E[H_n] as a quartic in m
    const float4 *ghc;       // FP32C compiled layouts: per GH cell the three float4 of gh_record
    R *pe, *pl;
    float *gp;
    const R *sh;             // spherical-harmonic node table
    const short *pmap;       // layout 1: set 1's cell of each pixel of set 0 (when aligned)
    unsigned *c_lo, *c_hi, *c_cnt;   // FP32C prior-cell sums / counts
    double *c_d;                     // FP64 prior-cell sums
    int *mmk;                        // FP32C range keys: min E, max E, max |L_z|
};

// Observable layouts compiled as straight-line code (set order, geometry,
// quantity); layout 0 walks the set descriptors at run time.
//   1: grid/mass + grid/GH            (pixels + IFU apertures)
//   2: shell/mass + annulus/GH        (shells + kinematic annuli)
//   3: shell/mass + annulus/mass + annulus/v_los^2
//   4: grid/mass + lookup-table/GH + lookup-table/GH (pixels + Voronoi-binned
//      IFU + long slit)
template <int V> using IC = std::integral_constant<int, V>;
template <int L, class F>
__device__ __forceinline__ void for_each_set(F &&f) {
    if constexpr (L == 1) {
        f(IC<0>{}, IC<M2M_GEOM_GRID>{}, IC<M2M_Q_MASS>{});
        f(IC<1>{}, IC<M2M_GEOM_GRID>{}, IC<M2M_Q_GH>{});
    } else if constexpr (L == 2) {
        f(IC<0>{}, IC<M2M_GEOM_SHELL>{}, IC<M2M_Q_MASS>{});
        f(IC<1>{}, IC<M2M_GEOM_ANNULUS>{}, IC<M2M_Q_GH>{});
    } else if constexpr (L == 3) {
        f(IC<0>{}, IC<M2M_GEOM_SHELL>{}, IC<M2M_Q_MASS>{});
        f(IC<1>{}, IC<M2M_GEOM_ANNULUS>{}, IC<M2M_Q_MASS>{});
        f(IC<2>{}, IC<M2M_GEOM_ANNULUS>{}, IC<M2M_Q_VLOS2>{});
    } else if constexpr (L == 4) {
        f(IC<0>{}, IC<M2M_GEOM_GRID>{}, IC<M2M_Q_MASS>{});
        f(IC<1>{}, IC<M2M_GEOM_LUT>{}, IC<M2M_Q_GH>{});
        f(IC<2>{}, IC<M2M_GEOM_LUT>{}, IC<M2M_Q_GH>{});
    }
}

// dot = sum_j K_j coef_j over the particle's cells, in set and moment order
template <class R, int L>
__device__ __forceinline__ R obs_dot(const PassArgs &a, const PassSmem<R> &S, R x, R y, R z,
                                     R X, R Ys, R vlos, bool cached, unsigned cc,
                                     long long i, long long epoch) {
    R dot = R(0);
    if constexpr (L == 0) {
        for (int k = 0; k < a.nsets; ++k) {
            const SetDev &s = a.sets[k];
            R Xk = X, Yk = Ys;
            if (s.psf) seeing<R>(s, k, i, epoch, Xk, Yk);
            int c = set_cell<R>(s, S.edges, x, y, z, Xk, Yk);
            if (c < 0) continue;
            int b = s.obs_off + c * s.nmom;
            if (s.quant == M2M_Q_MASS) {
                dot = dot + S.coef[b];
            } else if (s.quant == M2M_Q_VLOS2) {
                dot = dot + (vlos * vlos) * S.coef[b];
            } else {
                R u[5];
                gh_eval(vlos, S.gh + s.gh_off + 5 * c, u);
#pragma unroll
                for (int m = 0; m < 5; ++m) dot = dot + u[m] * S.coef[b + m];
            }
        }
    } else {
        int c0 = -1;     // set 0's cell
        for_each_set<L>([&](auto K, auto G, auto Q) {
            constexpr int k = decltype(K)::value, g = decltype(G)::value, q = decltype(Q)::value;
            const SetDev &s = a.sets[k];
            int c;
            if (cached) {
                c = (int)((cc >> s.cshift) & (unsigned)s.cmask) - 1;
            } else if (sizeof(R) == 4 && L == 1 && k == 1 && s.pmap_len) {
                c = c0 >= 0 ? (int)S.pmap[c0] : -1;                       // aligned with set 0's pixels
            } else {
                R Xk = X, Yk = Ys;
                if (L == 4 && s.psf) seeing<R>(s, k, i, epoch, Xk, Yk);   // seeing: lookup-table layout
                c = cell_t<R, g>(s, S.epair, x, y, z, Xk, Yk);
            }
            if (k == 0) c0 = c;
            if (c >= 0) {
                if constexpr (q == M2M_Q_MASS) {
                    dot = dot + S.coef[s.obs_off + c];
                } else if constexpr (q == M2M_Q_VLOS2) {
                    dot = dot + (vlos * vlos) * S.coef[s.obs_off + c];
                } else {
                    // sum_n coef_n u_n(nu) = exp(-nu m / 2) * P(m), m = nu c1,
                    // with the quartic P of this cell built in the prologue
                    if constexpr (sizeof(R) == 4) {
                        // the record of gh_record: the norm in the exponent
                        const float4 *r = S.ghc + 3 * (s.ghc_off + c);
                        const float4 g0 = r[0], g1 = r[1];
                        const float P4 = r[2].x;
                        const float dv = vlos - g0.x, m = dv * g0.y;
                        const float e = ex2_ftz(fmaf(dv * m, g0.z, g0.w));
                        float q = fmaf(P4, m, g1.w);
                        q = fmaf(q, m, g1.z);
                        q = fmaf(q, m, g1.y);
                        q = fmaf(q, m, g1.x);
                        dot = dot + e * q;
                    } else {
                        const R *g = S.gh + s.gh_off + 5 * c;
                        const R *P = S.gpoly + s.gh_off + 5 * c;
                        const R nu = (vlos - g[0]) * g[1];
                        const R m = nu * g[2];
                        const R e = gh_exp(R(-0.5) * nu * m);
                        R q = fma(P[4], m, P[3]);
                        q = fma(q, m, P[2]);
                        q = fma(q, m, P[1]);
                        q = fma(q, m, P[0]);
                        dot = dot + e * q;
                    }
                }
            }
        });
    }
    return dot;
}

// The update's Gauss-Hermite term of one cell, sum_n coef_n u_n(nu) =
// exp(-nu m / 2) P(m) with m = nu c1: the quartic P from the cell's
// coefficients cf0..cf4, t2 and norm (E[H_n] over N(m, t2) as polynomials
// in m, van der Marel & Franx H_0..H_4).
template <class R>
__device__ __forceinline__ void gh_quartic(R t2, R nrm, R cf0, R cf1, R cf2, R cf3, R cf4, R P[5]) {
    const R r2 = R(1.4142135623730951), r3 = R(1.7320508075688772), r24 = R(4.898979485566356);
    P[0] = nrm * (cf0 + cf2 * ((R(2) * t2 - R(1)) / r2) + cf4 * ((R(12) * t2 * t2 - R(12) * t2 + R(3)) / r24));
    P[1] = nrm * (cf1 * r2 + cf3 * ((R(6) * t2 - R(3)) / r3));
    P[2] = nrm * (cf2 * r2 + cf4 * ((R(24) * t2 - R(12)) / r24));
    P[3] = nrm * (cf3 * (R(2) / r3));
    P[4] = nrm * (cf4 * (R(4) / r24));
}

struct ThreadAcc {
    double s_d, w_d;     // FP64 path
    float s_f, w_f;      // FP32C path
    bool ovf, bad;
};

__device__ __forceinline__ void hist_add(const PassSmem<float> &S, int b, float v, float fs, int sh, ThreadAcc &t) {
    fx_red(S.hL, S.hM, S.hH, b, v, fs, sh, t.ovf);
}
__device__ __forceinline__ void hist_add(const PassSmem<double> &S, int b, double v, float, int, ThreadAcc &) {
    atomicAdd(S.h_d + b, v);
}

template <class R, int L>
__device__ __forceinline__ unsigned scatter(const PassArgs &a, const PassSmem<R> &S, R x, R y, R z,
                                            R X, R Ys, R vlos, R wv, float fs, ThreadAcc &ovf,
                                            long long i, long long epoch) {
    const int sh = a.fx_shift;
    unsigned packed = 0u;
    if constexpr (L == 0) {
        for (int k = 0; k < a.nsets; ++k) {
            const SetDev &s = a.sets[k];
            R Xk = X, Yk = Ys;
            if (s.psf) seeing<R>(s, k, i, epoch, Xk, Yk);
            int c = set_cell<R>(s, S.edges, x, y, z, Xk, Yk);
            if (c < 0) continue;
            int b = s.obs_off + c * s.nmom;
            if (s.quant == M2M_Q_MASS) {
                hist_add(S, b, wv, fs, sh, ovf);
            } else if (s.quant == M2M_Q_VLOS2) {
                hist_add(S, b, wv * (vlos * vlos), fs, sh, ovf);
            } else {
                R u[5];
                gh_eval(vlos, S.gh + s.gh_off + 5 * c, u);
#pragma unroll
                for (int m = 0; m < 5; ++m) hist_add(S, b + m, wv * u[m], fs, sh, ovf);
            }
        }
    } else {
        int c0 = -1;     // set 0's cell
        for_each_set<L>([&](auto K, auto G, auto Q) {
            constexpr int k = decltype(K)::value, g = decltype(G)::value, q = decltype(Q)::value;
            const SetDev &s = a.sets[k];
            R Xk = X, Yk = Ys;
            if (L == 4 && s.psf) seeing<R>(s, k, i, epoch, Xk, Yk);       // seeing: lookup-table layout
            int c;
            if (sizeof(R) == 4 && L == 1 && k == 1 && s.pmap_len)          // aligned with set 0's pixels
                c = c0 >= 0 ? (int)S.pmap[c0] : -1;
            else
                c = cell_t<R, g>(s, S.epair, x, y, z, Xk, Yk);
            if (k == 0) c0 = c;
            packed |= (unsigned)(c + 1) << s.cshift;
            if (c >= 0 && wv != R(0)) {
                if constexpr (q == M2M_Q_MASS || q == M2M_Q_VLOS2) {
                    const R v = q == M2M_Q_MASS ? wv : wv * (vlos * vlos);
                    if constexpr (sizeof(R) == 4) {
                        const float Sv = v * fs;
                        if (fabsf(Sv) < FX_FAST) fx_red_fast(S.hL, S.hM, s.obs_off + c, Sv);
                        else hist_add(S, s.obs_off + c, v, fs, sh, ovf);
                    } else {
                        hist_add(S, s.obs_off + c, v, fs, sh, ovf);
                    }
                } else {
                    const int b = s.obs_off + 5 * c;
                    if constexpr (sizeof(R) == 4) {
                        // |u_n| <= sqrt 2 for every n and nu (a Gaussian average
                        // of Hermite functions, Cramer's bound), so one test of
                        // the weight decides the fast path for all five terms,
                        // each added as soon as it is formed: (w 2^sh) u_n =
                        // (w u_n) 2^sh exactly
                        const float4 *rc = S.ghc + 3 * (s.ghc_off + c);
                        const float W = wv * fs;
                        if (fabsf(W) < 0.5f * FX_FAST) {
                            gh_red_stream(vlos, rc, W, S.hL, S.hM, b);
                        } else {
                            R u[5];
                            gh_eval_rec(vlos, rc, u);
#pragma unroll
                            for (int m = 0; m < 5; ++m) hist_add(S, b + m, wv * u[m], fs, sh, ovf);
                        }
                    } else {
                        R u[5];
                        gh_eval(vlos, S.gh + s.gh_off + 5 * c, u);
#pragma unroll
                        for (int m = 0; m < 5; ++m) hist_add(S, b + m, wv * u[m], fs, sh, ovf);
                    }
                }
            }
        });
    }
    return packed;
}

// expm1 for the small exponents of the weight update (|d| < 2^-7: Taylor
// to d^5, relative error < 2^-40), the library routine otherwise.
__device__ __forceinline__ float expm1_small(float d) {
    if (fabsf(d) < 0.0078125f) {
        float p = fmaf(d, 1.0f / 120.0f, 1.0f / 24.0f);
        p = fmaf(d, p, 1.0f / 6.0f);
        p = fmaf(d, p, 0.5f);
        p = fmaf(d, p, 1.0f);
        return d * p;
    }
    return expm1f(d);
}

// The weight update of one particle: returns the new weight; wnf = the new
// weight in the state precision (for the entropy and weight sums), L1 =
// ln(w_new/w_hat).  FP32C takes ln w_hat
// (kept per particle in float by the library), FP64 w_hat itself.
__device__ __forceinline__ double upd_weight(double w, float lnwh, float dot, const PassArgs &a, float &wnf, float &L1) {
    const float wf = d2f_fast(w);
    const float L = __logf(wf) - lnwh;
    const float G = a.f_mu * (-L - a.f_ent_c) - dot;
    const float d = a.f_eps_dt * G;
    const float e = expm1_small(d);
    const double wn = fma(w, f2d_fast(e), w);
    wnf = fmaf(wf, e, wf);
    L1 = L + d;
    return wn;
}
__device__ __forceinline__ double upd_weight(double w, double what, double dot, const PassArgs &a, double &wnd, double &L1) {
    double L = log(w / what);
    double G = a.mu * (-L - a.ent_c) - dot;
    double d = a.eps_dt * G;
    double wn = w * exp(d);
    wnd = wn;
    L1 = L + d;
    return wn;
}

__device__ __forceinline__ void acc_stats(ThreadAcc &t, float wnf, float L1) {
    t.s_f = fmaf(-wnf, L1, t.s_f);
    t.w_f += wnf;
}
__device__ __forceinline__ void acc_stats(ThreadAcc &t, double wnd, double L1) {
    t.s_d += -wnd * L1;
    t.w_d += wnd;
}
__device__ __forceinline__ float to_r(double v, float *) { return d2f_fast(v); }
__device__ __forceinline__ double to_r(double v, double *) { return v; }
__device__ __forceinline__ float rlog_ratio(double w, float lnwh, float *) { return __logf(d2f_fast(w)) - lnwh; }
__device__ __forceinline__ double rlog_ratio(double w, double what, double *) { return log(w / what); }

template <class R>
__device__ __forceinline__ void cell_add(const PassArgs &a, const PassSmem<R> &S, int c, double wv, bool &ovf);
template <>
__device__ __forceinline__ void cell_add<float>(const PassArgs &a, const PassSmem<float> &S, int c, double wv, bool &ovf) {
    long long q = d2fixed(wv, a.cell_shift, ovf);
    if (q) fixed_add(S.c_lo, S.c_hi, c, q);
    atomicAdd(S.c_cnt + c, 1u);
}
template <>
__device__ __forceinline__ void cell_add<double>(const PassArgs &a, const PassSmem<double> &S, int c, double wv, bool &) {
    atomicAdd(S.c_d + c, wv);
    atomicAdd((unsigned *)(S.c_lo) + c, 1u);
}

// FL != 0: the flags are that compile-time constant (specialised kernels of
// the steady-state step), else they come from the arguments.
template <class R, int L, int FL, int PK>
__device__ __forceinline__ void particle(const PassArgs &a, const PassSmem<R> &S, int i,
                                         R &x, R &y, R &z, R &vx, R &vy, R &vz, double &w, R what,
                                         unsigned cc, ThreadAcc &t, R &emin, R &emax, R &lzm, float fs,
                                         long long epoch, bool cache_read) {
    // what: FP32C ln w_hat, FP64 w_hat; epoch: pushes the positions have had
    // at the start of this pass; cache_read: cc holds the cells at x
    const int fl = FL ? FL : a.flags;
    const R sn = KC(R, a.sin_i, a.f_sin_i), cs = KC(R, a.cos_i, a.f_cos_i);
    double wn = w;
    // FP32C, a weight in the normal float range: the float arithmetic of
    // the update and the entropy on the two words of the double directly
    bool fast = false;
    if constexpr (sizeof(R) == 4) {
        const unsigned hi = (unsigned)__double2hiint(w), lo = (unsigned)__double2loint(w);
        fast = w_normal(hi);
        if (fast && (fl & (F_UPD | F_STATS))) {
            const float wf = w_to_float(hi, lo);
            if (fl & F_UPD) {
                const float vlos = vy * sn + vz * cs;
                const bool cached = L != 0 && cache_read;
                const float dot = obs_dot<R, L>(a, S, x, y, z, x, z * sn - y * cs, vlos, cached, cc, i, epoch);
                const float Lw = lg2_ftz(wf) * LN2F - what;
                const float G = a.f_mu * (-Lw - a.f_ent_c) - dot;
                const float d = a.f_eps_dt * G;
                const float e = expm1_small(d);
                wn = fma(w, (double)e, w);
                // negative (or -0), infinite or NaN
                if ((unsigned)__double2hiint(wn) >= 0x7FF00000u) t.bad = true;
                if (fl & F_STATS) acc_stats(t, fmaf(wf, e, wf), Lw + d);
            } else {
                acc_stats(t, wf, lg2_ftz(wf) * LN2F - what);
            }
        }
    }
    if ((fl & (F_UPD | F_STATS)) && !fast) {
        if (d_pos(w)) {
            R L1;
            R wr;
            if (fl & F_UPD) {
                R X = x, Ys = z * sn - y * cs, vlos = vy * sn + vz * cs;
                const bool cached = L != 0 && cache_read;
                R dot = obs_dot<R, L>(a, S, x, y, z, X, Ys, vlos, cached, cc, i, epoch);
                wn = upd_weight(w, what, dot, a, wr, L1);
                if (d_bad(wn)) t.bad = true;
            } else {
                wr = to_r(w, (R *)nullptr);
                L1 = rlog_ratio(w, what, (R *)nullptr);
            }
            if (fl & F_STATS) acc_stats(t, wr, L1);
        } else if (__double_as_longlong(w) != 0ll) {
            t.bad = true;       // negative, -0 or NaN weight
        }
    }
    if (fl & F_PUSH) kdk<R, PK>(x, y, z, vx, vy, vz, a, S.sh, i);
    if (fl & F_SCAT) {
        R X = x, Ys = z * sn - y * cs, vlos = vy * sn + vz * cs;
        // the scattered weight is a function of the stored (double) weight
        // alone, whichever pass applied the update
        R wv;
        if constexpr (sizeof(R) == 4) {
            // the truncated float in the normal range; 0 below it (d2f_fast
            // gives 0 there too); beyond it no term is representable
            const unsigned hn = (unsigned)__double2hiint(wn);
            wv = w_normal(hn) ? w_to_float(hn, (unsigned)__double2loint(wn)) : 0.f;
            if (hn - 0x47F00000u < 0x38000000u) t.ovf = true;   // 2^128 <= wn < inf
        } else {
            wv = to_r(wn, (R *)nullptr);
        }
        // the scatter sees the positions after this pass's push, if any
        const unsigned packed = scatter<R, L>(a, S, x, y, z, X, Ys, vlos, wv, fs, t, i,
                                              epoch + ((fl & F_PUSH) ? 1 : 0));
        // (a pass with its flags compiled in always belongs to a context
        // with a cell cache; the run-time-flag passes ask)
        if (L != 0 && (FL != 0 || a.cache_write)) a.cell_cache[i] = packed;
    }
    if (fl & F_MINMAX) {
        R E, Lz;
        energy_lz<R, PK>(x, y, z, vx, vy, vz, a, S.sh, E, Lz);
        if constexpr (sizeof(R) == 4) {
            // FP32C: the warp's min E, max E, max |L_z| as order-preserving
            // integer keys (one warp reduction each), then the block's by
            // shared-memory atomics: nothing carried across the particle loop
            const bool ok = E == E;
            const int kE = ok ? fkey((float)E) : 0;
            const float al = fabsf((float)Lz);
            const unsigned m = __activemask();
            const int r0 = __reduce_min_sync(m, ok ? kE : INT_MAX);
            const int r1 = __reduce_max_sync(m, ok ? kE : INT_MIN);
            const int r2 = __reduce_max_sync(m, al == al ? __float_as_int(al) : 0);
            if ((int)(threadIdx.x & 31) == __ffs(m) - 1) {
                atomicMin(S.mmk, r0);
                atomicMax(S.mmk + 1, r1);
                atomicMax(S.mmk + 2, r2);
            }
        } else {
            emin = fmin(emin, E);
            emax = fmax(emax, E);
            lzm = fmax(lzm, fabs(Lz));
        }
    }
    if (fl & F_CELLS) {
        int c = prior_cell<R, PK>(x, y, z, vx, vy, vz, a, S.pe, S.pl, S.gp, S.sh);
        a.cell_ids[i] = c;
        cell_add<R>(a, S, c, wn, t.ovf);
    }
    w = wn;
}

// Stage buffer of one block chunk (NT consecutive particles): x,y,z,vx,vy,vz
// (R), w, w_hat (double), cached cells (u32), each array contiguous.
template <class R, int NT> struct Chunk {
    static constexpr int OX = 0, OY = NT * sizeof(R), OZ = 2 * NT * sizeof(R), OVX = 3 * NT * sizeof(R),
                         OVY = 4 * NT * sizeof(R), OVZ = 5 * NT * sizeof(R), OW = 6 * NT * sizeof(R),
                         OWH = OW + 8 * NT, OCC = OWH + 8 * NT, BYTES = OCC + 4 * NT;
};
constexpr int PIPE_STAGES = 2;    // the pipeline below is written for two stages
// particles a block scatters between two flushes of its FP32C histogram
// (keeps every int32 part-sum of fx_red exact)
constexpr int FX_SEG = 32768;
// FP32C fixed-point resolution: 2^-FX_AVG_BITS of the average weight
constexpr int FX_AVG_BITS = 25;

// One block's share of a pass over the particles of one model: block `bid`
// of `nblk` blocks that share the model's particles (grid-stride).
template <class R, int NT, int L, int PIPE, int FL = 0, int PK = PK_ANY>
__device__ __forceinline__ void pass_body(const PassArgs &a, const int bid, const int nblk) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ __align__(8) unsigned long long bars[PIPE ? 2 * PIPE_STAGES : 1];   // full[], empty[]
    constexpr bool FX = sizeof(R) == 4;
    const int fl = FL ? FL : a.flags;
    PassSmem<R> S{};
    unsigned char *p = smem;
    const int nobs = a.nobs;
    if (fl & F_SCAT) {
        if (FX) { S.hL = (int *)p; S.hM = S.hL + nobs; S.hH = S.hM + nobs; p += 12 * ((nobs + 3) & ~3); }
        else { S.h_d = (double *)p; p += 8 * ((nobs + 1) & ~1); }
    }
    if (fl & F_UPD) { S.coef = (const R *)p; p += sizeof(R) * ((nobs + 3) & ~3); }
    S.edges = (const R *)p; p += sizeof(R) * ((a.edge_len + 3) & ~3);
    S.epair = (const Pair<R> *)p; p += 2 * sizeof(R) * ((a.edge_len + 1) & ~1);
    S.gh = (const R *)p; p += sizeof(R) * ((a.gh_len + 3) & ~3);
    constexpr bool GHC = FX && L != 0;      // combined GH records instead of gh + gpoly
    if (GHC) { S.ghc = (const float4 *)p; p += 48 * (a.gh_len / 5); }
    else if (fl & F_UPD) { S.gpoly = (const R *)p; p += sizeof(R) * ((a.gh_len + 3) & ~3); }
    if (FX && L == 1) { S.pmap = (const short *)p; p += 2 * ((a.sets[1].pmap_len + 7) & ~7); }
    const int sh_len = (a.sh_tab && (fl & (F_PUSH | F_MINMAX | F_CELLS))) ? a.sh_row * a.sh_K : 0;
    if (sh_len) { S.sh = (const R *)p; p += sizeof(R) * ((sh_len + 3) & ~3); }
    if (fl & F_CELLS) {
        S.pe = (R *)p; p += sizeof(R) * ((a.nE + 4) & ~3);
        S.pl = (R *)p; p += sizeof(R) * ((a.nL + 4) & ~3);
        S.gp = (float *)p; p += 16;
        if (FX) {
            S.c_lo = (unsigned *)p; S.c_hi = S.c_lo + a.ncells; S.c_cnt = S.c_hi + a.ncells;
            p += 12 * ((a.ncells + 3) & ~3);
        } else {
            S.c_d = (double *)p; p += 8 * ((a.ncells + 1) & ~1);
            S.c_lo = (unsigned *)p; p += 4 * ((a.ncells + 3) & ~3);   // counts
        }
    }
    unsigned char *stages = p;        // PIPE: PIPE_STAGES chunk buffers of NT particles
    if constexpr (PIPE) {
        if (threadIdx.x == 0) {
            for (int st = 0; st < PIPE_STAGES; ++st) {
                mbar_init(&bars[st], 1);                          // full: the producer's expect_tx
                mbar_init(&bars[PIPE_STAGES + st], NT / 32);      // empty: one arrival per warp
            }
            fence_mbar_init();
        }
    }
    // prologue: clear histograms, stage the tables (the edge and GH tables
    // are fixed at m2m_init; everything else a preceding kernel may write,
    // so it is read after griddep_wait)
    if (fl & F_SCAT) {
        unsigned *hz = FX ? (unsigned *)S.hL : (unsigned *)S.h_d;
        for (int k = threadIdx.x; k < (FX ? 3 : 2) * nobs; k += NT) hz[k] = 0u;
    }
    for (int k = threadIdx.x; k < a.edge_len; k += NT) {
        const R *et = (const R *)a.edge_tab;
        const R e0 = et[k], e1 = k + 1 < a.edge_len ? et[k + 1] : R(INFINITY);
        ((R *)S.edges)[k] = e0;
        Pair<R> pr;
        pr.x = e0;
        pr.y = e1;
        ((Pair<R> *)S.epair)[k] = pr;
    }
    stage<2>((R *)S.gh, (const R *)a.gh_tab, a.gh_len, threadIdx.x, NT);
    if (FX && L == 1) stage<1>((short *)S.pmap, a.sets[1].pmap, a.sets[1].pmap_len, threadIdx.x, NT);
    griddep_wait();
    if (fl & F_UPD) stage<4>((R *)S.coef, (const R *)a.coef, nobs, threadIdx.x, NT);
    if (sh_len) stage<4>((R *)S.sh, (const R *)a.sh_tab, sh_len, threadIdx.x, NT);
    if (L != 0 && (GHC || (fl & F_UPD))) {
        // E[H_n] over N(m, t2) as polynomials in m (van der Marel & Franx
        // H_0..H_4), weighted by this step's coefficients of the cell (0
        // in a pass without an update; FP32C keeps them with the cell's GH
        // parameters in one record)
        for (int k = 0; k < a.nsets; ++k) {
            const SetDev &st = a.sets[k];
            if (st.quant != M2M_Q_GH) continue;
            for (int c = threadIdx.x; c < st.ncell; c += NT) {
                const R *g = (const R *)a.gh_tab + st.gh_off + 5 * c;
                const R t2 = g[3], nrm = g[4];
                R P[5] = {R(0), R(0), R(0), R(0), R(0)};
                if (fl & F_UPD) {
                    const R *cf = (const R *)a.coef + st.obs_off + 5 * c;
                    // the compiled FP32C record carries the norm in its exponent
                    gh_quartic<R>(t2, GHC ? R(1) : nrm, cf[0], cf[1], cf[2], cf[3], cf[4], P);
                }
                if constexpr (GHC) {
                    float4 rec[3];
                    gh_record(g[0], g[1], g[2], t2, nrm, (const float *)P, rec);
                    float4 *rc = (float4 *)S.ghc + 3 * (st.ghc_off + c);
                    rc[0] = rec[0]; rc[1] = rec[1]; rc[2] = rec[2];
                } else {
                    R *Pd = (R *)S.gpoly + st.gh_off + 5 * c;
                    for (int q = 0; q < 5; ++q) Pd[q] = P[q];
                }
            }
        }
    }
    __shared__ int mmk[3];
    S.mmk = mmk;
    if ((fl & F_MINMAX) && threadIdx.x == 0) {
        mmk[0] = fkey(INFINITY); mmk[1] = fkey(-INFINITY); mmk[2] = 0;
    }
    if (fl & F_CELLS) {
        if (FX) {
            for (int k = threadIdx.x; k < 3 * a.ncells; k += NT) S.c_lo[k] = 0u;   // lo, hi, cnt
        } else {
            for (int k = threadIdx.x; k < a.ncells; k += NT) { S.c_d[k] = 0.0; S.c_lo[k] = 0u; }
        }
        prior_setup<R>(a, S.pe, S.pl, S.gp);
    }
    __syncthreads();

    ThreadAcc t{0.0, 0.0, 0.f, 0.f, false, false};
    R emin = R(INFINITY), emax = R(-INFINITY), lzm = R(0);
    const float fs = a.fx_shift <= 127 ? __int_as_float((a.fx_shift + 127) << 23) : INFINITY;
    const long long n = a.n;
    R *px = (R *)a.x, *py = (R *)a.y, *pz = (R *)a.z, *pvx = (R *)a.vx, *pvy = (R *)a.vy, *pvz = (R *)a.vz;
    const bool wr_pos = (fl & F_PUSH) != 0;
    const bool wr_w = (fl & F_UPD) != 0;
    const bool need_what = (fl & (F_UPD | F_STATS)) != 0;
    // FP32C reads ln w_hat (float, kept by the library), FP64 w_hat
    const R *pwh = FX ? (const R *)a.lnwhat : (const R *)a.what;
    const bool need_cc = L != 0 && a.cache_read && (fl & F_UPD);
    // FP32C histogram flush (all threads, after a barrier): the exact totals
    // H * 2^32 + M * 2^16 + L of this segment go into the global totals with
    // 64-bit integer atomics, or into this block's slot for the residual to
    // sum (integer sums: the result does not depend on the order).
    int nseg = 0;
    auto flush_hist = [&](bool last) {
        long long *sl = (long long *)a.slots + (long long)bid * nobs;
        for (int k = threadIdx.x; k < nobs; k += NT) {
            const long long v = (long long)(((unsigned long long)(long long)S.hH[k] << 32) +
                                            ((unsigned long long)(long long)S.hM[k] << 16) +
                                            (unsigned long long)(long long)S.hL[k]);
            if (!last) { S.hL[k] = 0; S.hM[k] = 0; S.hH[k] = 0; }
            if (a.fx_atomic) {
                if (v) atomicAdd(a.y_acc + k, (unsigned long long)v);
            } else {
                sl[k] = nseg ? sl[k] + v : v;
            }
        }
        ++nseg;
    };
    if constexpr (PIPE) {
        // block-level pipeline over chunks of NT consecutive particles
        // (chunk c of this block's grid stride): thread 0 stages the chunk
        // of the next iteration into the other stage with one bulk copy per
        // array (>= 4 KB each) once every warp has read that stage's
        // previous chunk (empty barrier); each thread takes its particle of
        // the current chunk from shared memory.  Every wait is bounded; a
        // wait that runs out records M2M_ERR_TIMEOUT and the loop goes on
        // (results invalid) so that the block's barriers stay matched.
        using C = Chunk<R, NT>;
        unsigned long long *full = bars, *empty = bars + PIPE_STAGES;
        const int lane = threadIdx.x & 31;
        const int nfull = (int)(n / NT), nch = (int)((n + NT - 1) / NT);
        const unsigned bytes = 6 * NT * sizeof(R) + 8 * NT + (need_what ? NT * sizeof(R) : 0) + (need_cc ? 4 * NT : 0);
        // thread 0: copies issued to / seen complete in stage 0 and 1 (scalars:
        // no local-memory array)
        int iss0 = 0, iss1 = 0, seen0 = 0, seen1 = 0;
        bool late = false;
        auto issue = [&](int c, int st) {    // thread 0 only
            if (c >= nfull) return;
            unsigned char *d = stages + st * C::BYTES;
            unsigned long long *b = full + st;
            if (st) ++iss1; else ++iss0;
            mbar_expect_tx(b, bytes);
            const size_t oR = (size_t)c * NT * sizeof(R), oD = (size_t)c * NT * 8, oC = (size_t)c * NT * 4;
            bulk_g2s(d + C::OX, (const char *)px + oR, NT * sizeof(R), b);
            bulk_g2s(d + C::OY, (const char *)py + oR, NT * sizeof(R), b);
            bulk_g2s(d + C::OZ, (const char *)pz + oR, NT * sizeof(R), b);
            bulk_g2s(d + C::OVX, (const char *)pvx + oR, NT * sizeof(R), b);
            bulk_g2s(d + C::OVY, (const char *)pvy + oR, NT * sizeof(R), b);
            bulk_g2s(d + C::OVZ, (const char *)pvz + oR, NT * sizeof(R), b);
            bulk_g2s(d + C::OW, (const char *)a.w + oD, NT * 8, b);
            if (need_what) bulk_g2s(d + C::OWH, (const char *)pwh + oR, NT * sizeof(R), b);
            if (need_cc) bulk_g2s(d + C::OCC, (const char *)a.cell_cache + oC, NT * 4, b);
        };
        __syncthreads();                     // barrier initialisation visible to all
        if (threadIdx.x == 0) {
            issue(bid, 0);
            issue(bid + nblk, 1);
        }
        int it = 0, k = 0;
        for (int c = bid; c < nch; c += nblk, ++k) {
            const int st = k & 1;
            const unsigned par = (unsigned)(k >> 1) & 1u;
            if (threadIdx.x == 0 && k >= 1 && c + nblk < nfull) {
                // the next iteration's chunk goes where the previous one was
                const int sp = (k + 1) & 1;
                if (mbar_wait(empty + sp, (unsigned)((k - 1) >> 1) & 1u)) issue(c + nblk, sp);
                else late = true;
            }
            const int i = c * NT + threadIdx.x;
            R x = R(0), y = R(0), z = R(0), vx = R(0), vy = R(0), vz = R(0);
            double w = 0.0;
            R wh = R(0);
            unsigned cc = 0u;
            if (c < nfull) {
                if (mbar_wait(full + st, par)) {
                    if (threadIdx.x == 0) { if (st) ++seen1; else ++seen0; }
                } else {
                    late = true;
                }
                const unsigned char *d = stages + st * C::BYTES;
                const int q = threadIdx.x;
                x = ((const R *)(d + C::OX))[q]; y = ((const R *)(d + C::OY))[q];
                z = ((const R *)(d + C::OZ))[q]; vx = ((const R *)(d + C::OVX))[q];
                vy = ((const R *)(d + C::OVY))[q]; vz = ((const R *)(d + C::OVZ))[q];
                w = ((const double *)(d + C::OW))[q];
                if (need_what) wh = ((const R *)(d + C::OWH))[q];
                if (need_cc) cc = ((const unsigned *)(d + C::OCC))[q];
                __syncwarp();
                if (lane == 0) mbar_arrive(empty + st);
            } else if (i < (int)n) {
                x = px[i]; y = py[i]; z = pz[i]; vx = pvx[i]; vy = pvy[i]; vz = pvz[i];
                w = a.w[i];
                if (need_what) wh = pwh[i];
                if (need_cc) cc = a.cell_cache[i];
            }
            if (i < (int)n) {
                particle<R, L, FL, PK>(a, S, i, x, y, z, vx, vy, vz, w, wh, cc, t, emin, emax, lzm, fs, a.epoch,
                                       a.cache_read != 0);
                if (wr_pos) {
                    __stcs(px + i, x); __stcs(py + i, y); __stcs(pz + i, z);
                    __stcs(pvx + i, vx); __stcs(pvy + i, vy); __stcs(pvz + i, vz);
                }
                if (wr_w) __stcs(a.w + i, w);
            }
            if (FX && (fl & F_SCAT) && ++it == FX_SEG / NT && c + nblk < nch) {
                __syncthreads();
                flush_hist(false);
                __syncthreads();
                it = 0;
            }
        }
        if (late) {
            atomicOr(a.err, ERR_TIMEOUT);
            // let copies still in flight land before the block exits
            if (threadIdx.x == 0) {
                for (int u = seen0; u < iss0; ++u)
                    if (!mbar_wait(full, (unsigned)u & 1u)) break;
                for (int u = seen1; u < iss1; ++u)
                    if (!mbar_wait(full + 1, (unsigned)u & 1u)) break;
            }
        }
    } else {
        // grid-stride over the particles with the next particle's state
        // loaded before the current one is processed; the trip count is the
        // same for every thread of the block, so the histograms can be
        // flushed (block-wide) every FX_SEG iterations
        const int stride = nblk * NT;
        int i = bid * NT + threadIdx.x;
        R x = R(0), y = R(0), z = R(0), vx = R(0), vy = R(0), vz = R(0);
        double w = 0.0;
        R wh = R(0);
        unsigned cc = 0u;
        if (i < (int)n) {
            x = __ldcs(px + i); y = __ldcs(py + i); z = __ldcs(pz + i);
            vx = __ldcs(pvx + i); vy = __ldcs(pvy + i); vz = __ldcs(pvz + i);
            w = __ldcs(a.w + i);
            if (need_what) wh = __ldcs(pwh + i);
            if (need_cc) cc = a.cell_cache[i];
        }
        int it = 0;
#pragma unroll 2
        for (int base = bid * NT; base < (int)n; base += stride, i += stride) {
            const int j = i + stride;
            R nx = R(0), ny = R(0), nz = R(0), nvx = R(0), nvy = R(0), nvz = R(0);
            double nw = 0.0;
            R nwh = R(0);
            unsigned ncc = 0u;
            if (j < (int)n) {
                nx = __ldcs(px + j); ny = __ldcs(py + j); nz = __ldcs(pz + j);
                nvx = __ldcs(pvx + j); nvy = __ldcs(pvy + j); nvz = __ldcs(pvz + j);
                nw = __ldcs(a.w + j);
                if (need_what) nwh = __ldcs(pwh + j);
                if (need_cc) ncc = a.cell_cache[j];
            }
            if (i < (int)n) {
                particle<R, L, FL, PK>(a, S, i, x, y, z, vx, vy, vz, w, wh, cc, t, emin, emax, lzm, fs, a.epoch,
                                       a.cache_read != 0);
                if (wr_pos) {
                    __stcs(px + i, x); __stcs(py + i, y); __stcs(pz + i, z);
                    __stcs(pvx + i, vx); __stcs(pvy + i, vy); __stcs(pvz + i, vz);
                }
                if (wr_w) __stcs(a.w + i, w);
            }
            x = nx; y = ny; z = nz; vx = nvx; vy = nvy; vz = nvz; w = nw; wh = nwh; cc = ncc;
            if (FX && (fl & F_SCAT) && ++it == FX_SEG / NT && base + stride < (int)n) {
                __syncthreads();
                flush_hist(false);
                __syncthreads();
                it = 0;
            }
        }
    }
    if (a.rec_pending) {
        // the record of the preceding step, by the first block to get here
        __shared__ int s_rec;
        if (threadIdx.x == 0) s_rec = atomicAdd(a.rec_ticket, 1ull) == a.rec_base;
        __syncthreads();
        if (s_rec && threadIdx.x < 32)
            record_warp(a.rec_chi, a.rec_chi_nblk, a.rec_stat, a.rec_stat_nblk, a.mu, a.rec_step, a.rec_write_ring,
                        (m2m_record *)a.ring, (m2m_record *)a.last, a.err);
    }
    griddep_launch();
    __syncthreads();
    // epilogue: flush the block-private histograms and partial sums
    if (fl & F_SCAT) {
        if (FX) {
            flush_hist(true);
        } else {
            double *sl = (double *)a.slots + (long long)bid * nobs;
            for (int k = threadIdx.x; k < nobs; k += NT) sl[k] = S.h_d[k];
        }
    }
    if (fl & F_CELLS) {
        if (FX) {
            for (int k = threadIdx.x; k < a.ncells; k += NT) {
                unsigned cn = S.c_cnt[k];
                if (cn) {
                    long long v = (long long)(((unsigned long long)S.c_hi[k] << 32) | (unsigned long long)S.c_lo[k]);
                    atomicAdd((unsigned long long *)a.cell_acc + k, (unsigned long long)v);
                    atomicAdd(a.cell_cnt + k, cn);
                }
            }
        } else {
            for (int k = threadIdx.x; k < a.ncells; k += NT) {
                unsigned cn = S.c_lo[k];
                if (cn) {
                    atomicAdd((double *)a.cell_acc + k, S.c_d[k]);
                    atomicAdd(a.cell_cnt + k, cn);
                }
            }
        }
    }
    if (fl & F_STATS) {
        double s_tot = 0.0, w_tot = 0.0;
        if (FX) {
            __shared__ float red2[128];
            block_sum2_ff(t.s_f, t.w_f, red2, s_tot, w_tot);
        } else {
            s_tot = block_sum(t.s_d, red);
            w_tot = block_sum(t.w_d, red);
        }
        if (threadIdx.x == 0) {
            a.stat_slots[2 * bid] = s_tot;
            a.stat_slots[2 * bid + 1] = w_tot;
        }
    }
    if ((fl & F_MINMAX) && FX) {
        __syncthreads();
        if (threadIdx.x == 0) {
            R *o = (R *)a.mm_slots + 4 * bid;
            o[0] = fkey_inv(S.mmk[0]); o[1] = fkey_inv(S.mmk[1]); o[2] = __int_as_float(S.mmk[2]); o[3] = R(0);
        }
    } else if (fl & F_MINMAX) {
        __shared__ R mm[3][32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            emin = fmin(emin, __shfl_xor_sync(0xffffffffu, emin, o));
            emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
            lzm = fmax(lzm, __shfl_xor_sync(0xffffffffu, lzm, o));
        }
        int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
        if (lane == 0) { mm[0][wp] = emin; mm[1][wp] = emax; mm[2][wp] = lzm; }
        __syncthreads();
        if (threadIdx.x == 0) {
            R e0 = mm[0][0], e1 = mm[1][0], l2 = mm[2][0];
            for (int k = 1; k < NT / 32; ++k) {
                e0 = fmin(e0, mm[0][k]); e1 = fmax(e1, mm[1][k]); l2 = fmax(l2, mm[2][k]);
            }
            R *o = (R *)a.mm_slots + 4 * bid;
            o[0] = e0; o[1] = e1; o[2] = l2; o[3] = R(0);
        }
    }
    if (t.ovf) atomicOr(a.err, ERR_OVERFLOW);
    if (t.bad) atomicOr(a.err, ERR_NONFINITE);
}

template <class R, int NT, int MINB, int L, int PIPE, int FL = 0, int PK = PK_ANY>
__global__ void __launch_bounds__(NT, MINB) k_pass(const __grid_constant__ PassArgs a) {
    pass_body<R, NT, L, PIPE, FL, PK>(a, blockIdx.x, gridDim.x);
}

// flags of the steady-state step pass: pending update, push, scatter, stats
constexpr int F_STEADY = F_UPD | F_PUSH | F_SCAT | F_STATS;

// Many models in one launch: block b runs block blk_rank[b] of
// blk_count[m] blocks of model m = blk_model[b]; each model's arguments are
// its own PassArgs (device array), the flags and cache use are shared.
struct BatchPass {
    const PassArgs *models;
    const int *blk_model, *blk_rank, *blk_count;
    int flags, cache_read, cache_write;
};
template <class R, int NT, int MINB, int L, int FL = 0, int PK = PK_ANY>
__global__ void __launch_bounds__(NT, MINB) k_pass_batch(const __grid_constant__ BatchPass b) {
    const int m = b.blk_model[blockIdx.x];
    __shared__ __align__(16) PassArgs a;
    static_assert(sizeof(PassArgs) % 4 == 0, "PassArgs copied as words");
    const unsigned *src = (const unsigned *)(b.models + m);
    for (int k = threadIdx.x; k < (int)(sizeof(PassArgs) / 4); k += NT) ((unsigned *)&a)[k] = src[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        a.flags = b.flags;
        a.cache_read = b.cache_read;
        a.cache_write = b.cache_write;
    }
    __syncthreads();
    pass_body<R, NT, L, 0, FL, PK>(a, b.blk_rank[blockIdx.x], b.blk_count[m]);
}

// ------------------------------------------------------------- residual
struct ResArgs {
    const void *slots; int nblk; int nobs; int fixed; double q;
    unsigned long long *y_acc; int fx_atomic;
    const double *Y, *inv_sigma;    // 1/sigma_j, 0 where sigma_j <= 0 (masked)
    double *Dt, *y, *Delta, *coef_d; void *coef_r; int r_float;
    int mode; double alpha, mu;
    const double *stat_slots; int stat_nblk;
    double *chi_slots; unsigned *ticket;
    m2m_record *ring, *last; long long rec_step; int write_ring;
    int tail;                       // 1: the last block writes the record; 0: the next pass does
    int *err;
};

// Eq. 1 for observable j with total yv: Delta_j = (y_j - Y_j)/sigma_j, the
// smoothed Delta~_j (mode 1: alpha Delta + (1 - alpha) Delta~; 2: Delta; 0:
// unchanged) and the update's coefficient Delta~_j/sigma_j (0 where the
// observable is masked); returns the chi^2 terms Delta~^2, Delta^2, |Delta~|.
__device__ __forceinline__ void residual_obs(const ResArgs &a, int j, double yv, double &c2, double &c2r,
                                             double &mx) {
    const double is = a.inv_sigma[j];
    const bool valid = is > 0.0;
    const double D = valid ? (yv - a.Y[j]) * is : 0.0;
    const double dold = a.Dt[j];
    const double dn = (a.mode == 1) ? a.alpha * D + (1.0 - a.alpha) * dold : (a.mode == 2 ? D : dold);
    const double cf = valid ? dn * is : 0.0;
    a.y[j] = yv;
    a.Delta[j] = D;
    if (a.mode != 0) a.Dt[j] = dn;
    a.coef_d[j] = cf;
    if (a.r_float) ((float *)a.coef_r)[j] = (float)cf;
    else ((double *)a.coef_r)[j] = cf;
    c2 = dn * dn; c2r = D * D; mx = fabs(dn);
}

#ifdef M2M_COMMON_KERNELS

// Deterministic strided sum over the block: thread k adds k, k+NT, ... in
// order, then a fixed shuffle tree.
__device__ __forceinline__ double block_sum_strided(const double *v, int stride, int off, int cnt, double *red) {
    double s = 0.0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) s += v[(long long)k * stride + off];
    return block_sum(s, red);
}

// FP32C (fx_atomic): one thread per observable in small blocks; the totals
// are exact integers already summed by the pass's atomics (re-zeroed here
// for the next scatter).  Slots (FP64, or FP32C without atomics): 32
// observables per block (lane = observable), the warps split the per-block
// slots with four independent accumulators each, in a fixed order.  The
// per-observable arithmetic is FP64 (slow on this part), so it is spread
// over many blocks; divisions by sigma are multiplications by its
// reciprocal.  Chi^2 partials per block, then the last block to finish
// writes the record.
constexpr int RES_NT = 1024;      // slot reduction
constexpr int RES_NT_FX = 128;    // FP32C atomic totals
__device__ __forceinline__ void residual_body(const ResArgs &a, const int bid, const int nblk) {
    griddep_wait();            // the totals of the preceding pass
    griddep_launch();          // the next pass may stage its fixed tables meanwhile
    constexpr int NW = RES_NT / 32;
    __shared__ unsigned long long si[NW][32];
    __shared__ double sd[NW][32];
    __shared__ double wred[3][NW];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const bool direct = a.fixed && a.fx_atomic;
    const int j = direct ? bid * blockDim.x + threadIdx.x : bid * 32 + lane;
    bool have = false;
    double yv = 0.0;
    if (direct) {
        if (j < a.nobs) {
            const unsigned long long tot = a.y_acc[j];
            a.y_acc[j] = 0ull;
            yv = (double)(long long)tot * a.q;
            have = true;
        }
    } else {
        if (j < a.nobs) {
            if (a.fixed) {
                const long long *sl = (const long long *)a.slots + j;
                unsigned long long acc[4] = {0, 0, 0, 0};
                int b = wp;
                for (; b + 3 * nw < a.nblk; b += 4 * nw) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[u] += (unsigned long long)sl[(long long)(b + u * nw) * a.nobs];
                }
                for (; b < a.nblk; b += nw) acc[0] += (unsigned long long)sl[(long long)b * a.nobs];
                si[wp][lane] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
            } else {
                const double *sl = (const double *)a.slots + j;
                double acc[4] = {0, 0, 0, 0};
                int b = wp;
                for (; b + 3 * nw < a.nblk; b += 4 * nw) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[u] += sl[(long long)(b + u * nw) * a.nobs];
                }
                for (; b < a.nblk; b += nw) acc[0] += sl[(long long)b * a.nobs];
                sd[wp][lane] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
            }
        }
        __syncthreads();
        if (wp == 0 && j < a.nobs) {
            if (a.fixed) {
                unsigned long long tot = 0;
                for (int k = 0; k < nw; ++k) tot += si[k][lane];
                yv = (double)(long long)tot * a.q;
            } else {
                for (int k = 0; k < nw; ++k) yv += sd[k][lane];
            }
            have = true;
        }
    }
    double c2 = 0.0, c2r = 0.0, mx = 0.0;
    if (have) residual_obs(a, j, yv, c2, c2r, mx);
    c2 = warp_sum(c2);
    c2r = warp_sum(c2r);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) { wred[0][wp] = c2; wred[1][wp] = c2r; wred[2][wp] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < nw; ++k) { s0 += wred[0][k]; s1 += wred[1][k]; s2 = fmax(s2, wred[2][k]); }
        a.chi_slots[3 * bid] = s0;
        a.chi_slots[3 * bid + 1] = s1;
        a.chi_slots[3 * bid + 2] = s2;
        if (a.tail) {
            __threadfence();
            s_last = (atomicAdd(a.ticket, 1u) == (unsigned)nblk - 1u);
        }
    }
    if (!a.tail) return;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < 32)
        record_warp(a.chi_slots, nblk, a.stat_slots, a.stat_nblk, a.mu, a.rec_step, a.write_ring, a.ring, a.last, a.err);
    if (threadIdx.x == 0) *a.ticket = 0u;
}

// The record of a step whose residual left it to the next pass, when no
// pass follows (one warp).
__global__ void k_record(const double *chi, int nch, const double *st, int nst, double mu, long long step,
                         int write_ring, m2m_record *ring, m2m_record *last, int *err) {
    griddep_wait();
    record_warp(chi, nch, st, nst, mu, step, write_ring, ring, last, err);
}

__global__ void __launch_bounds__(RES_NT) k_residual(const __grid_constant__ ResArgs a) {
    residual_body(a, blockIdx.x, gridDim.x);
}

// Residuals of many models in one launch (FP32C totals: one thread per
// observable); per-model arguments in a device array, step fields shared.
struct BatchRes {
    const ResArgs *models;
    const int *blk_model, *blk_rank, *blk_count;
    int mode, write_ring;
    long long rec_step;           // added to *step (records stay right when a graph replays)
    const long long *step;
};
__global__ void __launch_bounds__(RES_NT_FX) k_residual_batch(const __grid_constant__ BatchRes b) {
    const int m = b.blk_model[blockIdx.x];
    __shared__ __align__(16) ResArgs a;
    static_assert(sizeof(ResArgs) % 4 == 0, "ResArgs copied as words");
    const unsigned *src = (const unsigned *)(b.models + m);
    for (int k = threadIdx.x; k < (int)(sizeof(ResArgs) / 4); k += blockDim.x) ((unsigned *)&a)[k] = src[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        a.mode = b.mode;
        a.write_ring = b.write_ring;
        a.rec_step = b.rec_step + *b.step;
    }
    __syncthreads();
    residual_body(a, b.blk_rank[blockIdx.x], b.blk_count[m]);
}

// 1/sigma_j (0 where sigma_j <= 0: masked observable)
__global__ void k_inv_sigma(const double *sigma, double *isig, int nobs) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nobs) isig[j] = sigma[j] > 0.0 ? 1.0 / sigma[j] : 0.0;
}

// ----------------------------------------------------------- prior means
// mean[c] = sum[c] / count[c]; then w_hat_i = mean[cell_i].
__global__ void k_prior_mean(const void *acc, const unsigned *cnt, int ncells, int fixed, double q, double *mean) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    unsigned k = cnt[c];
    double s = fixed ? (double)((const long long *)acc)[c] * q : ((const double *)acc)[c];
    mean[c] = k ? s / (double)k : 0.0;
}

__global__ void k_prior_gather(const int *cell, const double *mean, double *what, float *lnwhat, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double m = mean[cell[i]];
        what[i] = m;
        if (lnwhat) lnwhat[i] = logf(__double2float_rn(m));
    }
}

// ln w_hat in float from w_hat (FP32C: read by the weight update).
__global__ void k_lnwhat(const double *what, float *lnwhat, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        lnwhat[i] = logf(__double2float_rn(what[i]));
}

// ------------------------------------------------------ spherical harmonics
// The expansion of the weighted particles (kind 4): per radial side j (side
// 0: r < r_0; side j: r_(j-1) <= r < r_j; r >= r_(K-1) left out), sums of
//   A terms  w P_l(mu) (r/r_j)^l             (j = 0..K-1)
//   B terms  w P_l(mu) (r_(j-1)/r)^(l+1)     (j = 1..K-1)
// each at most w in size; the table kernel multiplies back r_j^l and
// r_(j-1)^-(l+1) in double.  FP32C: the float terms are summed exactly in
// 64-bit fixed point (one scale serves every side; its resolution, 2^-56 of
// the total weight, is far below a float term's rounding).  FP64: double
// sums (block-private, then global atomics), since a 64-bit fixed point
// would round double terms of large N far above their own precision.
struct ShArgs {
    const void *x, *y, *z;
    const double *w;
    long long n;
    int K;
    const void *e2;                 // R[K] squared node radii (float: smallest float >= the double)
    const void *rn, *irn;           // R[K] node radii and their reciprocals
    int gmode; float ga, gb;        // index guess for e2
    int sh;                         // fixed point: value * 2^sh
    unsigned long long *sum;        // [10][K]: A_l sides (l = 0..8 even), then B_l sides
    int *err;
};

__device__ __forceinline__ long long to_fixed(float v, int sh, bool &ovf) { return f2fixed(v, sh, ovf); }
__device__ __forceinline__ long long to_fixed(double v, int sh, bool &ovf) { return d2fixed(v, sh, ovf); }

template <class R>
__global__ void __launch_bounds__(512) k_sh_coef(const __grid_constant__ ShArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool FX = sizeof(R) == 4;
    const int K = a.K, NS = 10 * K;
    unsigned *lo = (unsigned *)smem, *hi = lo + NS;     // FX: (lo, hi) pairs; else NS doubles
    double *acc = (double *)smem;
    R *e2 = (R *)(hi + NS), *rn = e2 + K, *irn = rn + K;
    for (int k = threadIdx.x; k < 2 * NS; k += blockDim.x) lo[k] = 0u;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        e2[k] = ((const R *)a.e2)[k];
        rn[k] = ((const R *)a.rn)[k];
        irn[k] = ((const R *)a.irn)[k];
    }
    __syncthreads();
    bool ovf = false, bad = false;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (shuffles)
    for (long long base = (long long)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const long long i = base + threadIdx.x;
        int j = K;
        long long q[10];           // FX: fixed-point terms
        R v[10];                   // double terms
#pragma unroll
        for (int m = 0; m < 10; ++m) { q[m] = 0; v[m] = R(0); }
        if (i < a.n) {
            const R x = ((const R *)a.x)[i], y = ((const R *)a.y)[i], z = ((const R *)a.z)[i];
            const double wd = a.w[i];
            const R r2 = (x * x + y * y) + z * z;
            if (r2 < e2[0]) {
                j = 0;
            } else {
                const int c = find_bin<R>(r2, e2, K - 1, a.gmode, a.ga, a.gb);
                j = c < 0 ? K : c + 1;                  // NaN or r >= r_(K-1): left out
            }
            if (d_bad(wd) && __double_as_longlong(wd) != 0ll) bad = true;
            if (j < K && d_pos(wd)) {
                const R wr = to_r(wd, (R *)nullptr);
                const R r = sqrt(r2);
                const R mu = r2 > R(0) ? z / r : R(0);
                R P[5], dP[5];
                legendre_even<R>(mu, P, dP);
                const R rho = r * irn[j], rho2 = rho * rho;
                R t = wr;
#pragma unroll
                for (int n = 0; n < 5; ++n) {
                    v[n] = t * P[n];
                    t = t * rho2;
                }
                if (j > 0) {
                    const R sg = rn[j - 1] / r, sg2 = sg * sg;
                    R u = wr * sg;
#pragma unroll
                    for (int n = 0; n < 5; ++n) {
                        v[5 + n] = u * P[n];
                        u = u * sg2;
                    }
                }
                if (FX)
#pragma unroll
                    for (int m = 0; m < 10; ++m) q[m] = to_fixed(v[m], a.sh, ovf);
            }
        }
        const int j0 = __shfl_sync(0xffffffffu, j, 0);
        if (__all_sync(0xffffffffu, j == j0)) {
            if (j0 < K) {
                // one side for the whole warp: warp sums, then one update
#pragma unroll
                for (int m = 0; m < 10; ++m) {
                    if (FX) {
                        long long u = q[m];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
                        q[m] = u;
                    } else {
                        v[m] = warp_sum(v[m]);
                    }
                }
                if (lane == 0)
#pragma unroll
                    for (int m = 0; m < 10; ++m) {
                        if (FX) { if (q[m]) fixed_add(lo, hi, m * K + j0, q[m]); }
                        else if (v[m] != R(0)) atomicAdd(acc + m * K + j0, (double)v[m]);
                    }
            }
        } else if (j < K) {
#pragma unroll
            for (int m = 0; m < 10; ++m) {
                if (FX) { if (q[m]) fixed_add(lo, hi, m * K + j, q[m]); }
                else if (v[m] != R(0)) atomicAdd(acc + m * K + j, (double)v[m]);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NS; k += blockDim.x) {
        if (FX) {
            const unsigned long long u = ((unsigned long long)hi[k] << 32) | lo[k];
            if (u) atomicAdd(a.sum + k, u);
        } else if (acc[k] != 0.0) {
            atomicAdd((double *)a.sum + k, acc[k]);
        }
    }
    if (ovf) atomicOr(a.err, ERR_OVERFLOW);
    if (bad) atomicOr(a.err, ERR_NONFINITE);
}

// Node tables from the side sums (one block): scale back, prefix sums for
// A_l(r_k) = sum_{j <= k}, suffix sums (outside in) for B_l(r_k) =
// sum_{j > k}, then F_l, D_l and the slopes to the next node, in double.
template <class R>
__global__ void k_sh_tables(const long long *sum, int K, const double *rn, double q, R *tab, int *err) {
    extern __shared__ __align__(16) double sd[];
    double *S = sd;                // [10][K] side sums, then A, B at the nodes
    double *FD = sd + 10 * K;      // [10][K] F_l, D_l at the nodes
    for (int k = threadIdx.x; k < 10 * K; k += blockDim.x) {
        const int m = k / K, j = k - m * K, n = m % 5, l = 2 * n;
        const double v = sizeof(R) == 4 ? (double)sum[k] * q : ((const double *)sum)[k];
        double s = 1.0;
        if (m < 5) {
            for (int e = 0; e < l; ++e) s *= rn[j];                       // r_j^l
        } else if (j > 0) {
            for (int e = 0; e <= l; ++e) s *= rn[j - 1];                  // r_(j-1)^(l+1)
            s = 1.0 / s;
        } else {
            s = 0.0;
        }
        S[k] = v * s;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double *row = S + threadIdx.x * K;
        double acc = 0.0;
        if (threadIdx.x < 5) {
            for (int k = 0; k < K; ++k) { acc += row[k]; row[k] = acc; }
        } else {
            for (int k = K - 1; k >= 0; --k) { const double b = row[k]; row[k] = acc; acc += b; }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double r = rn[k], ir = 1.0 / r;
        double rl = 1.0;           // r^l
        for (int n = 0; n < 5; ++n) {
            const int l = 2 * n;
            const double A = S[n * K + k], B = S[(5 + n) * K + k];
            const double irl1 = ir / rl;                  // r^-(l+1)
            FD[n * K + k] = A * irl1 + B * rl;
            FD[(5 + n) * K + k] = -(double)(l + 1) * A * (irl1 * ir) + (l > 0 ? (double)l * B * (rl * ir) : 0.0);
            rl = rl * r * r;
        }
        if (!isfinite(FD[k])) atomicOr(err, ERR_NONFINITE);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        R *row = tab + (size_t)k * SH_ROW;
        const bool last = k == K - 1;
        const double h = last ? 1.0 : 1.0 / (rn[k + 1] - rn[k]);
        for (int n = 0; n < 5; ++n) {
            const double F = FD[n * K + k], D = FD[(5 + n) * K + k];
            row[n] = (R)F;
            row[10 + n] = (R)D;
            row[5 + n] = last ? R(0) : (R)((FD[n * K + k + 1] - F) * h);
            row[15 + n] = last ? R(0) : (R)((FD[(5 + n) * K + k + 1] - D) * h);
        }
        row[20] = (R)rn[k];
    }
}

// The expansions with m != 0 (kinds 5 and 6, basis B): per radial side j,
// for each of its NT terms t, A terms w Y_t (r/r_j)^l and B terms
// w Y_t (r_(j-1)/r)^(l+1) (j > 0), each at most 1.7 w in size, summed exactly
// in 64-bit fixed point (FP32C) or in double (FP64) as for the axisymmetric
// expansion; [2 NT][K] side sums, row t for A and NT + t for B.  The terms
// are generated one at a time; a warp whose particles share one side adds
// warp sums.
template <class B, class R>
__global__ void __launch_bounds__(512) k_ex_coef(const __grid_constant__ ShArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool FX = sizeof(R) == 4;
    constexpr int NT = B::NT;
    const int K = a.K, NS = 2 * NT * K;
    unsigned *lo = (unsigned *)smem, *hi = lo + NS;
    double *acc = (double *)smem;
    R *e2 = (R *)(hi + NS), *rn = e2 + K, *irn = rn + K;
    for (int k = threadIdx.x; k < 2 * NS; k += blockDim.x) lo[k] = 0u;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        e2[k] = ((const R *)a.e2)[k];
        rn[k] = ((const R *)a.rn)[k];
        irn[k] = ((const R *)a.irn)[k];
    }
    __syncthreads();
    bool ovf = false, bad = false;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (shuffles)
    for (long long base = (long long)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const long long i = base + threadIdx.x;
        int j = K;
        R mu = R(1), nx = R(0), ny = R(0), ta[5], tb[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) { ta[n] = R(0); tb[n] = R(0); }
        if (i < a.n) {
            const R x = ((const R *)a.x)[i], y = ((const R *)a.y)[i], z = ((const R *)a.z)[i];
            const double wd = a.w[i];
            const R r2 = (x * x + y * y) + z * z;
            if (r2 < e2[0]) {
                j = 0;
            } else {
                const int c = find_bin<R>(r2, e2, K - 1, a.gmode, a.ga, a.gb);
                j = c < 0 ? K : c + 1;                  // NaN or r >= r_(K-1): left out
            }
            if (d_bad(wd) && __double_as_longlong(wd) != 0ll) bad = true;
            if (j < K && d_pos(wd)) {
                const R wr = to_r(wd, (R *)nullptr);
                const R r = sqrt(r2), ir = r2 > R(0) ? R(1) / r : R(0);
                nx = x * ir; ny = y * ir;
                mu = r2 > R(0) ? z * ir : R(1);
                // w (r/r_j)^l and w (r_(j-1)/r)^(l+1) for the basis's l
                const R rho = r * irn[j], sg = j > 0 ? rn[j - 1] * ir : R(0);
                const R rs = B::LSTEP == 2 ? rho * rho : rho, ss = B::LSTEP == 2 ? sg * sg : sg;
                ta[0] = wr;
                tb[0] = wr * sg;
#pragma unroll
                for (int n = 1; n < 5; ++n) { ta[n] = ta[n - 1] * rs; tb[n] = tb[n - 1] * ss; }
            } else {
                j = j < K ? K + 1 : j;      // a particle of zero weight adds nothing
            }
        }
        const int j0 = __shfl_sync(0xffffffffu, j, 0);
        const bool same = __all_sync(0xffffffffu, j == j0);
        ex_terms<B, R>(mu, nx, ny, [&](int t, int l, int m, R c, R q0, R q1, R C, R gx, R gy) {
            const R Y = c * q0 * C;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const R v = (side == 0 ? ta[B::slot(l)] : tb[B::slot(l)]) * Y;
                const int row = side * NT + t;
                if (same) {
                    if (j0 < K) {
                        if (FX) {
                            long long u = to_fixed(v, a.sh, ovf);
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
                            if (lane == 0 && u) fixed_add(lo, hi, row * K + j0, u);
                        } else {
                            const R u = warp_sum(v);
                            if (lane == 0 && u != R(0)) atomicAdd(acc + row * K + j0, (double)u);
                        }
                    }
                } else if (j < K && v != R(0)) {
                    if (FX) {
                        const long long u = to_fixed(v, a.sh, ovf);
                        if (u) fixed_add(lo, hi, row * K + j, u);
                    } else {
                        atomicAdd(acc + row * K + j, (double)v);
                    }
                }
            }
        });
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NS; k += blockDim.x) {
        if (FX) {
            const unsigned long long u = ((unsigned long long)hi[k] << 32) | lo[k];
            if (u) atomicAdd(a.sum + k, u);
        } else if (acc[k] != 0.0) {
            atomicAdd((double *)a.sum + k, acc[k]);
        }
    }
    if (ovf) atomicOr(a.err, ERR_OVERFLOW);
    if (bad) atomicOr(a.err, ERR_NONFINITE);
}

// F_t and D_t at node k from the node sums A (rows 0..NT-1) and B (rows
// NT..2NT-1) held in S ([2NT][K]), with the 4 pi/(2l+1) of the addition
// theorem.
template <class B>
__device__ __forceinline__ void ex_node_FD(const double *S, int K, const double *rn, int k, int t, double &F,
                                           double &D) {
    const int l = B::l_of(t);
    const double r = rn[k], ir = 1.0 / r;
    double rl = 1.0;
    for (int e = 0; e < l; ++e) rl *= r;                           // r^l
    const double A = S[t * K + k], Bs = S[(B::NT + t) * K + k];
    const double c = 12.566370614359172 / (double)(2 * l + 1);     // 4 pi/(2l+1)
    const double irl1 = ir / rl;                                   // r^-(l+1)
    F = c * (A * irl1 + Bs * rl);
    D = c * (-(double)(l + 1) * A * (irl1 * ir) + (l > 0 ? (double)l * Bs * (rl * ir) : 0.0));
}

// Node tables of an expansion with m != 0 from its side sums (one block):
// scale back, prefix sums (A) and suffix sums (B), then F_t, D_t and the
// slopes to the next node.
template <class B, class R>
__global__ void k_ex_tables(const long long *sum, int K, const double *rn, double q, R *tab, int *err) {
    extern __shared__ __align__(16) double sd[];
    constexpr int NT = B::NT, NR = 2 * NT, ROW = B::ROW;
    double *S = sd;                // [2NT][K] side sums, then A, B at the nodes
    for (int k = threadIdx.x; k < NR * K; k += blockDim.x) {
        const int row = k / K, j = k - row * K, t = row % NT, l = B::l_of(t);
        const double v = sizeof(R) == 4 ? (double)sum[k] * q : ((const double *)sum)[k];
        double s = 1.0;
        if (row < NT) {
            for (int e = 0; e < l; ++e) s *= rn[j];                       // r_j^l
        } else if (j > 0) {
            for (int e = 0; e <= l; ++e) s *= rn[j - 1];                  // r_(j-1)^(l+1)
            s = 1.0 / s;
        } else {
            s = 0.0;
        }
        S[k] = v * s;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        double *row = S + threadIdx.x * K;
        double acc = 0.0;
        if (threadIdx.x < NT) {
            for (int k = 0; k < K; ++k) { acc += row[k]; row[k] = acc; }
        } else {
            for (int k = K - 1; k >= 0; --k) { const double b = row[k]; row[k] = acc; acc += b; }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        R *row = tab + (size_t)k * ROW;
        const bool last = k == K - 1;
        const double h = last ? 1.0 : 1.0 / (rn[k + 1] - rn[k]);
        bool fin = true;
        for (int t = 0; t < NT; ++t) {
            double F, D, F1 = 0.0, D1 = 0.0;
            ex_node_FD<B>(S, K, rn, k, t, F, D);
            if (!last) ex_node_FD<B>(S, K, rn, k + 1, t, F1, D1);
            fin = fin && isfinite(F) && isfinite(D);
            row[t] = (R)F;
            row[2 * NT + t] = (R)D;
            row[NT + t] = last ? R(0) : (R)((F1 - F) * h);
            row[3 * NT + t] = last ? R(0) : (R)((D1 - D) * h);
        }
        row[4 * NT] = (R)rn[k];
        if (!fin) atomicOr(err, ERR_NONFINITE);
    }
}

#endif  // M2M_COMMON_KERNELS

// ------------------------------------------------------------- k_cells
template <class R>
__global__ void k_cells(const __grid_constant__ PassArgs a, int *obs_cells, int *prior_cells) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *p = smem;
    R *edges = (R *)p; p += sizeof(R) * ((a.edge_len + 3) & ~3);
    R *pe = (R *)p; p += sizeof(R) * ((a.nE + 4) & ~3);
    R *pl = (R *)p; p += sizeof(R) * ((a.nL + 4) & ~3);
    float *gp = (float *)p;
    for (int k = threadIdx.x; k < a.edge_len; k += blockDim.x) edges[k] = ((const R *)a.edge_tab)[k];
    if (prior_cells) prior_setup<R>(a, pe, pl, gp);
    __syncthreads();
    R s = KC(R, a.sin_i, a.f_sin_i), c = KC(R, a.cos_i, a.f_cos_i);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        R x = ((const R *)a.x)[i], y = ((const R *)a.y)[i], z = ((const R *)a.z)[i];
        R vx = ((const R *)a.vx)[i], vy = ((const R *)a.vy)[i], vz = ((const R *)a.vz)[i];
        R X = x, Ys = z * s - y * c;
        for (int k = 0; k < a.nsets; ++k) {
            R Xk = X, Yk = Ys;
            if (a.sets[k].psf) seeing<R>(a.sets[k], k, i, a.epoch, Xk, Yk);
            obs_cells[(long long)k * a.n + i] = set_cell<R>(a.sets[k], edges, x, y, z, Xk, Yk);
        }
        if (prior_cells) prior_cells[i] = prior_cell<R>(x, y, z, vx, vy, vz, a, pe, pl, gp, (const R *)a.sh_tab);
    }
}

// Kernel tables, one per precision, each in its own translation unit.
void *pass_kernel_f32(int threads, int layout);
void *pass_kernel_f32_pipe(int layout);
void *pass_kernel_f32_steady(int layout, int pk = PK_ANY);
void *pass_kernel_f32_compiled(int flags, int layout, int pk);   // NULL if not compiled
void *pass_kernel_f32_pipe_steady(int layout);
void *pass_kernel_f32_batch(int layout, bool steady = false, int pk = PK_ANY);
void *steps_kernel_f32(int layout, int pk);                      // NULL if not compiled
void *pass_kernel_f64(int threads, int layout);
void *cells_kernel_f32();
void *cells_kernel_f64();

// Text returned by m2m_last_error(NULL) (errors not tied to a context).
void note_context_free_error(const char *msg);

}  // namespace m2m
