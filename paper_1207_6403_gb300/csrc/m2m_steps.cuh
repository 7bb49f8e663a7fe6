// Persistent multi-step kernel of the FP32C step (compiled observable
// layouts and potential signatures).
//
// One cooperative launch advances the model by several M2M steps (Section 2
// of the paper: push, scatter, residual, weight update), one block per SM,
// each block holding a fixed contiguous range of particles for the whole
// launch.  Per step:
//   1. the block's particles: the weight update pending from the previous
//      step's residual (at x_t), the KDK push to x_{t+1}, the scatter into
//      the block's shared-memory histogram, the entropy / weight partials
//      (and, on a launch's last step when the priors are due, the (E, L_z)
//      range);
//   2. the histogram into the int64 observable totals (integer atomics);
//   3. grid barrier;
//   4. the residual (Eq. 1 with the smoothing): each block takes a slice of
//      the observables, reads and clears their totals, writes Delta,
//      Delta~ and the update's coefficients, and leaves its chi^2 partials;
//   5. grid barrier; one warp writes the step record while the next
//      step's particles run.
// The arithmetic is that of k_pass and k_residual (the same particle and
// residual functions), so the state after a launch equals, bit for bit,
// the state after the same steps taken as one pass and one residual launch
// each (integer histogram sums do not depend on their order).  What it
// saves is the gap between the launches: the residual's launch and
// completion, the next pass's table staging, and the tail of a grid-stride
// pass whose blocks end at different times.
#pragma once
#include "m2m_kernels.cuh"

namespace m2m {

struct StepsArgs {
    PassArgs p;                   // particles, tables, potential, observables (flags unused)
    ResArgs r;                    // residual: totals, targets, 1/sigma, Delta~, outputs (mode 1)
    long long nsteps;             // steps of this launch, >= 1
    long long t0;                 // steps taken before the launch (records t0+1 ...)
    long long epoch0;             // pushes the positions have had at the launch
    int first_upd;                // the first step applies the pending weight update
    int first_cache;              // the cell cache holds the cells of the current positions
    int last_range;               // the last step also takes the (E, L_z) range
    unsigned long long *bar;      // grid-barrier arrivals, zero at launch
    double *st2;                  // [2][grid][2]: S, sum w of each block, by step parity
    double *chi2;                 // [2][grid][3]: chi^2, sum Delta^2, max |Delta~|, by step parity
    long long wait_ns;            // limit of one barrier wait (globaltimer ns)
    int test_stall;               // test only: block 0 never arrives at the first barrier
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch (every block resident): each
// block arrives once on a monotonic counter and waits until `target`
// arrivals have been counted.  The block's writes before the barrier are
// published by the release of its arrival (after the block-wide barrier)
// and seen by the acquiring loads of the waiting blocks.  The wait is
// bounded by wait_ns of the globaltimer: a wait that runs out records
// ERR_TIMEOUT and the block goes on (the launch's results are then
// invalid), so no block waits forever.
__device__ __forceinline__ void grid_barrier(unsigned long long *bar, unsigned long long target, long long wait_ns,
                                             int *err, bool arrive = true) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) red_release_add_u64(bar, 1ull);
        if (ld_acquire_u64(bar) < target) {
            const unsigned long long t0 = globaltimer_ns();
            for (;;) {
                if (ld_acquire_u64(bar) >= target) break;
                if ((long long)(globaltimer_ns() - t0) > wait_ns) {
                    atomicOr(err, ERR_TIMEOUT);
                    break;
                }
            }
        }
    }
    __syncthreads();
}

// One step's particles of a block.  The particles are taken in warp chunks
// of 32 consecutive ones, dealt to the warps of the grid in a fixed order:
// chunk c goes to warp (c mod 32G) (warp w of block b being number
// w G + b), so every block holds particles from the whole array (the arrays
// are often ordered by radius, and a contiguous range would give one block
// the crowded centre and another the empty outskirts) and the blocks'
// counts differ by at most one chunk per warp.  Every warp of a block runs
// the block's largest chunk count (a warp past its last chunk idles), so
// the histogram flushes that keep its part-sums exact stay block-uniform.
// The next chunk's state is loaded before the current one is processed.
template <int L, int PK, int FL>
__device__ __forceinline__ void steps_particles(const PassArgs &a, const PassSmem<float> &S, int G, int nit,
                                                ThreadAcc &t, float fs, long long epoch, bool cache_read) {
    constexpr int NT = 1024;
    float *px = (float *)a.x, *py = (float *)a.y, *pz = (float *)a.z;
    float *pvx = (float *)a.vx, *pvy = (float *)a.vy, *pvz = (float *)a.vz;
    const bool need_cc = (FL & F_UPD) && cache_read;
    // 32-bit indices: n < 2^31, so i + stride stays below 2^32
    const unsigned n = (unsigned)a.n, stride = (unsigned)G * NT;
    float emin = 0.f, emax = 0.f, lzm = 0.f;       // unused (FP32C range: shared-memory keys)
    unsigned i = ((threadIdx.x >> 5) * (unsigned)G + blockIdx.x) * 32u + (threadIdx.x & 31);
    float x = 0.f, y = 0.f, z = 0.f, vx = 0.f, vy = 0.f, vz = 0.f, wh = 0.f;
    double w = 0.0;
    unsigned cc = 0u;
    // every array is addressed by the same byte offset from its base (4-
    // and 8-byte elements), so one offset per element size serves them all
    if (i < n) {
        const size_t o4 = (size_t)i * 4u, o8 = (size_t)i * 8u;
        x = __ldcs(at(px, o4)); y = __ldcs(at(py, o4)); z = __ldcs(at(pz, o4));
        vx = __ldcs(at(pvx, o4)); vy = __ldcs(at(pvy, o4)); vz = __ldcs(at(pvz, o4));
        w = __ldcs(at(a.w, o8));
        wh = __ldcs(at(a.lnwhat, o4));
        if (need_cc) cc = *at(a.cell_cache, o4);
    }
    int it = 0;
#pragma unroll 2
    for (int k = 0; k < nit; ++k, i += stride) {
        const unsigned j = i + stride;
        float nx = 0.f, ny = 0.f, nz = 0.f, nvx = 0.f, nvy = 0.f, nvz = 0.f, nwh = 0.f;
        double nw = 0.0;
        unsigned ncc = 0u;
        if (j < n) {
            const size_t o4 = (size_t)j * 4u, o8 = (size_t)j * 8u;
            nx = __ldcs(at(px, o4)); ny = __ldcs(at(py, o4)); nz = __ldcs(at(pz, o4));
            nvx = __ldcs(at(pvx, o4)); nvy = __ldcs(at(pvy, o4)); nvz = __ldcs(at(pvz, o4));
            nw = __ldcs(at(a.w, o8));
            nwh = __ldcs(at(a.lnwhat, o4));
            if (need_cc) ncc = *at(a.cell_cache, o4);
        }
        if (i < n) {
            particle<float, L, FL, PK>(a, S, (int)i, x, y, z, vx, vy, vz, w, wh, cc, t, emin, emax, lzm, fs, epoch,
                                       cache_read);
            const size_t o4 = (size_t)i * 4u, o8 = (size_t)i * 8u;
            __stcs(at(px, o4), x); __stcs(at(py, o4), y); __stcs(at(pz, o4), z);
            __stcs(at(pvx, o4), vx); __stcs(at(pvy, o4), vy); __stcs(at(pvz, o4), vz);
            if (FL & F_UPD) __stcs(at(a.w, o8), w);
        }
        x = nx; y = ny; z = nz; vx = nvx; vy = nvy; vz = nvz; w = nw; wh = nwh; cc = ncc;
        if (++it == FX_SEG / NT && k + 1 < nit) {
            // keep every part-sum of the histogram exact (at most FX_SEG
            // terms per bin between flushes): this segment into the int64
            // totals
            __syncthreads();
            for (int q = threadIdx.x; q < a.nobs; q += NT) {
                const long long v = (long long)(((unsigned long long)(long long)S.hH[q] << 32) +
                                                ((unsigned long long)(long long)S.hM[q] << 16) +
                                                (unsigned long long)(long long)S.hL[q]);
                S.hL[q] = 0; S.hM[q] = 0; S.hH[q] = 0;
                if (v) atomicAdd(a.y_acc + q, (unsigned long long)v);
            }
            __syncthreads();
            it = 0;
        }
    }
}

// Dynamic shared memory: that of the steady pass of the same layout
// (pass_smem_bytes with the steady flags).
template <int L, int PK>
__global__ void __launch_bounds__(1024, 1) k_steps(const __grid_constant__ StepsArgs A) {
    constexpr int NT = 1024;
    using R = float;
    const PassArgs &a = A.p;
    const ResArgs &r = A.r;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[96];
    __shared__ float redf[128];
    __shared__ int mmk[3];
    PassSmem<R> S{};
    unsigned char *p = smem;
    const int nobs = a.nobs, nobs4 = (nobs + 3) & ~3;
    // the histogram's three parts each 16-byte aligned (vector flushes)
    S.hL = (int *)p; S.hM = S.hL + nobs4; S.hH = S.hM + nobs4; p += 12 * nobs4;
    S.coef = (const R *)p; p += 4 * nobs4;
    S.edges = (const R *)p; p += 4 * ((a.edge_len + 3) & ~3);
    S.epair = (const Pair<R> *)p; p += 8 * ((a.edge_len + 1) & ~1);
    S.gh = (const R *)p; p += 4 * ((a.gh_len + 3) & ~3);
    S.ghc = (const float4 *)p; p += 48 * (a.gh_len / 5);
    if (L == 1) { S.pmap = (const short *)p; p += 2 * ((a.sets[1].pmap_len + 7) & ~7); }
    S.mmk = mmk;

    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    // chunk iterations of this block (its warp 0 has the most chunks)
    const long long nch = (a.n + 31) / 32, gw = 32ll * G;
    const int nit = (int)((nch - b + gw - 1) / gw);
    // the block's observables in the residual
    const int j0 = (int)((long long)nobs * b / G), j1 = (int)((long long)nobs * (b + 1) / G);
    const bool vec = (nobs & 3) == 0;       // coefficients readable as float4

    // fixed tables, once per launch
    for (int k = threadIdx.x; k < a.edge_len; k += NT) {
        const R *et = (const R *)a.edge_tab;
        ((R *)S.edges)[k] = et[k];
        Pair<R> pr;
        pr.x = et[k];
        pr.y = k + 1 < a.edge_len ? et[k + 1] : R(INFINITY);
        ((Pair<R> *)S.epair)[k] = pr;
    }
    for (int k = threadIdx.x; k < a.gh_len; k += NT) ((R *)S.gh)[k] = ((const R *)a.gh_tab)[k];
    if (L == 1)
        for (int k = threadIdx.x; k < a.sets[1].pmap_len; k += NT) ((short *)S.pmap)[k] = a.sets[1].pmap[k];
    if (threadIdx.x == 0) { mmk[0] = fkey(INFINITY); mmk[1] = fkey(-INFINITY); mmk[2] = 0; }

    const float fs = a.fx_shift <= 127 ? __int_as_float((a.fx_shift + 127) << 23) : INFINITY;
    unsigned long long round = 0;
    bool ovf = false, bad = false;
    for (long long s = 0; s < A.nsteps; ++s) {
        const bool upd = s > 0 || A.first_upd;
        const bool rng = A.last_range && s == A.nsteps - 1;
        const bool cache_read = s > 0 || A.first_cache;
        const long long epoch = A.epoch0 + s;
        const int par = (int)((A.t0 + s) & 1);
        // this step's coefficients (the previous step's residual wrote them
        // during this launch: read past L1); the histogram cleared while
        // they arrive
        if (upd) {
            if (vec) {
                for (int k = threadIdx.x; k < nobs / 4; k += NT)
                    ((float4 *)S.coef)[k] = __ldcg((const float4 *)r.coef_r + k);
            } else {
                for (int k = threadIdx.x; k < nobs; k += NT) ((R *)S.coef)[k] = __ldcg((const R *)r.coef_r + k);
            }
        }
        for (int k = threadIdx.x; k < 3 * nobs4 / 4; k += NT) ((int4 *)S.hL)[k] = make_int4(0, 0, 0, 0);
        __syncthreads();
        // the GH records of this step's update
        for (int k = 0; k < a.nsets; ++k) {
            const SetDev &st = a.sets[k];
            if (st.quant != M2M_Q_GH) continue;
            for (int c = threadIdx.x; c < st.ncell; c += NT) {
                const R *g = S.gh + st.gh_off + 5 * c;
                const R t2 = g[3], nrm = g[4];
                R P[5] = {R(0), R(0), R(0), R(0), R(0)};
                if (upd) {
                    const R *cf = S.coef + st.obs_off + 5 * c;
                    gh_quartic<R>(t2, R(1), cf[0], cf[1], cf[2], cf[3], cf[4], P);   // the norm: in the exponent
                }
                float4 rec[3];
                gh_record(g[0], g[1], g[2], t2, nrm, P, rec);
                float4 *rc = (float4 *)S.ghc + 3 * (st.ghc_off + c);
                rc[0] = rec[0]; rc[1] = rec[1]; rc[2] = rec[2];
            }
        }
        __syncthreads();

        // the previous step's record, by the last warp of the grid (the one
        // with the fewest particles) before its particles: its FP64 sums run
        // beside the other warps' particle work (the partials stay in place
        // until the next step's residual)
        if (s > 0 && b == G - 1 && wp == NT / 32 - 1)
            record_warp(A.chi2 + (size_t)3 * (par ^ 1) * G, G, A.st2 + (size_t)2 * (par ^ 1) * G, G, r.mu, A.t0 + s,
                        1, r.ring, r.last, a.err);
        ThreadAcc t{0.0, 0.0, 0.f, 0.f, false, false};
        if (upd) {
            if (rng) steps_particles<L, PK, F_STEADY | F_MINMAX>(a, S, G, nit, t, fs, epoch, cache_read);
            else steps_particles<L, PK, F_STEADY>(a, S, G, nit, t, fs, epoch, cache_read);
        } else {
            if (rng) steps_particles<L, PK, F_PUSH | F_SCAT | F_STATS | F_MINMAX>(a, S, G, nit, t, fs, epoch, cache_read);
            else steps_particles<L, PK, F_PUSH | F_SCAT | F_STATS>(a, S, G, nit, t, fs, epoch, cache_read);
        }
        ovf |= t.ovf;
        bad |= t.bad;
        // the entropy and weight partials: each warp's in float-float
        float sh = t.s_f, sl = 0.f, wh = t.w_f, wl = 0.f;
        warp_ff2(sh, sl, wh, wl);
        if (lane == 0) { redf[wp] = sh; redf[32 + wp] = sl; redf[64 + wp] = wh; redf[96 + wp] = wl; }
        __syncthreads();
        if (wp == 0) {
            // the block's, in the same float-float tree over the warps
            sh = redf[lane]; sl = redf[32 + lane]; wh = redf[64 + lane]; wl = redf[96 + lane];
            warp_ff2(sh, sl, wh, wl);
            if (lane == 0) {
                A.st2[(size_t)2 * (par * G + b)] = (double)sh + (double)sl;
                A.st2[(size_t)2 * (par * G + b) + 1] = (double)wh + (double)wl;
                if (rng) {
                    float *o = (float *)a.mm_slots + 4 * b;
                    o[0] = fkey_inv(mmk[0]); o[1] = fkey_inv(mmk[1]); o[2] = __int_as_float(mmk[2]); o[3] = 0.f;
                }
            }
        } else {
            // meanwhile the other warps flush the histogram into the int64
            // totals (integer atomics: any order; a warp's 32 atomics on 32
            // consecutive totals, two cache lines)
            for (int k = (int)threadIdx.x - 32; k < nobs; k += NT - 32) {
                const long long v = (long long)(((unsigned long long)(long long)S.hH[k] << 32) +
                                                ((unsigned long long)(long long)S.hM[k] << 16) +
                                                (unsigned long long)(long long)S.hL[k]);
                if (v) atomicAdd(a.y_acc + k, (unsigned long long)v);
            }
        }
        round += (unsigned long long)G;
        grid_barrier(A.bar, round, A.wait_ns, a.err, !(A.test_stall && b == 0 && s == 0));

        // residual of the block's observables, one thread each: read and
        // clear their totals
        double c2 = 0.0, c2r = 0.0, mx = 0.0;
        for (int j = j0 + (int)threadIdx.x; j < j1; j += NT) {
            const unsigned long long tot = atomicExch(a.y_acc + j, 0ull);
            double e2 = 0.0, e2r = 0.0, emx = 0.0;
            residual_obs(r, j, (double)(long long)tot * r.q, e2, e2r, emx);
            c2 += e2; c2r += e2r; mx = fmax(mx, emx);
        }
        // the chi^2 partials of the warps that had observables (the first
        // two unless a block has more than 64)
        const int nwa = min(NT / 32, (j1 - j0 + 31) / 32);
        if (wp < nwa) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c2 += __shfl_xor_sync(0xffffffffu, c2, o);
                c2r += __shfl_xor_sync(0xffffffffu, c2r, o);
                mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (lane == 0) { red[3 * wp] = c2; red[3 * wp + 1] = c2r; red[3 * wp + 2] = mx; }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int k = 0; k < nwa; ++k) { s0 += red[3 * k]; s1 += red[3 * k + 1]; s2 = fmax(s2, red[3 * k + 2]); }
            double *o = A.chi2 + (size_t)3 * (par * G + b);
            o[0] = s0; o[1] = s1; o[2] = s2;
        }
        round += (unsigned long long)G;
        grid_barrier(A.bar, round, A.wait_ns, a.err);
    }
    // the launch's last record
    if (b == G - 1 && wp == 0) {
        const int par = (int)((A.t0 + A.nsteps - 1) & 1);
        record_warp(A.chi2 + (size_t)3 * par * G, G, A.st2 + (size_t)2 * par * G, G, r.mu, A.t0 + A.nsteps, 1,
                    r.ring, r.last, a.err);
    }
    if (ovf) atomicOr(a.err, ERR_OVERFLOW);
    if (bad) atomicOr(a.err, ERR_NONFINITE);
}

}  // namespace m2m
