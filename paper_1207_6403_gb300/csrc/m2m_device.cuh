// Device-side building blocks of the M2M step (sm_103a).
//
// Everything that decides an integer (bin and cell membership) or feeds one
// (the orbit push) is evaluated in the state precision R with a fixed
// operation order and no contraction (the library is compiled with
// -fmad=false; fmaf/fma are written out only where rounding order does not
// matter).  Membership is "edge_j <= v < edge_{j+1}" against edge tables
// that, for R = float, hold the smallest float >= each double edge, which is
// exactly the same test as comparing against the double edge.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace m2m {

constexpr int MAXSETS = 4;
constexpr int MAXPOT = 4;
constexpr int MAXOBS = 8192;
constexpr int MAXCELLS = 16385;

enum { F_UPD = 1, F_PUSH = 2, F_SCAT = 4, F_STATS = 8, F_MINMAX = 16, F_CELLS = 32 };
enum { G_LIN = 0, G_LOG = 1, G_BIS = 2 };
enum { ERR_NONFINITE = 1, ERR_OVERFLOW = 2, ERR_TIMEOUT = 4 };

struct SetDev {
    int geom, quant, nx, ny, nmom;
    int ncell;            // cells of the set (nx*ny pixels of a grid, nx shells or annuli, the LUT's apertures)
    int obs_off;          // first observable of this set
    int ex_off, ey_off;   // offsets into the edge table
    int gh_off;           // offset into the GH table (5 values per cell)
    int ghc_off;          // the same in cells (gh_off / 5)
    int gx_mode, gy_mode; // index guess for the x / y edges
    float gx_a, gx_b, gy_a, gy_b;
    float gx_top, gy_top; // nx - 1, ny - 1 as floats (clamp of the guess)
    int cshift, cmask;    // packed cell cache: ((cell + 1) & cmask) << cshift
    const int *lut;       // geometry 4: device table of nx*ny cell ids (-1: none)
    const void *psf;      // seeing: 2^bits displacement quantiles (state precision), or null
    int psf_shift;        // 32 - bits
    unsigned psf_seed;    // key word 0 of the draws
    // a grid set whose every edge is an edge of the grid of set 0 (as the
    // floats the cells are decided against): its cell as a function of set
    // 0's pixel, from a table of set 0's nx*ny pixels (-1: none); 0 = off
    int pmap_len;
    const short *pmap;
};

struct PotDev {
    int kind;             // 1 hernquist, 2 nfw, 3 log, 4 spherical harmonics
    int ik;               // sh: number of radial nodes K
    double c[6];          // hernquist: GM, a;  log: Rc2, iq2, v0sq, hv;  nfw: C=4 pi rho_s r_s^3, r_s, 1/r_s
                          // sh: -, r_0, r_(K-1), lgc = (K-1)/log2(r_(K-1)/r_0), -lgc log2(r_0), 1/r_0
    float cf[6];          // the same rounded once to float (no per-particle conversions)
};

// Spherical-harmonic node table: one row of SH_ROW values per radial node k
// (0..K-1), in the state precision:
//   [0..4]   F_l(r_k)          l = 0, 2, 4, 6, 8
//   [5..9]   dF_l per unit r to node k+1 (slope of the linear interpolant)
//   [10..14] D_l(r_k)  (= dF_l/dr at the node)
//   [15..19] slope of D_l to node k+1
//   [20]     r_k
// The last row has zero slopes.
constexpr int SH_ROW = 21;
constexpr int SH_MAXK = 512;

struct PassArgs {
    void *x, *y, *z, *vx, *vy, *vz;
    double *w, *what;
    const float *lnwhat;                    // FP32C: ln w_hat per particle (library-owned)
    long long n;
    long long epoch;                        // pushes the positions have had at the pass's start
    int flags;
    int nsets, nobs, npot;
    SetDev sets[MAXSETS];
    PotDev pot[MAXPOT];
    double eps_dt, mu, ent_c, hdt, dt, sin_i, cos_i;
    float f_eps_dt, f_mu, f_ent_c, f_hdt, f_dt, f_sin_i, f_cos_i, f_pk, f_pgma;
    const void *edge_tab; int edge_len;     // R
    const void *gh_tab;   int gh_len;       // R, 5 per GH cell: V, 1/S, c1, t2, norm
    const void *coef;                       // R[nobs]
    void *slots;                            // FP64: [grid][nobs] double per-block sums
    unsigned long long *y_acc;              // FP32C: [nobs] int64 fixed-point totals
    int fx_atomic;                          // FP32C: flush to y_acc with atomics (else slots)
    int fx_shift;                           // fixed point: value * 2^fx_shift
    int cell_shift;                         // FP32C prior-cell sums: weight * 2^cell_shift
    double *stat_slots;                     // [grid][2]: S, sum w
    // priors
    int prior_kind, nE, nL, ncells;
    double pk, pgma;                        // e_lc: a/GM, GM*a
    void *mm_slots; int mm_nblocks;         // [mm_nblocks][4] R: min E, max E, max|Lz|, pad
    const void *sh_tab; int sh_K, sh_row;   // expansion node table (R, sh_row values per node) or NULL
    void *facc; int facc_read;              // expansion potentials: force at the positions (R, [3][n]) or NULL
    // record of the preceding step, left by its residual to this pass (the
    // first block to finish its particles writes it; see record_warp)
    int rec_pending, rec_write_ring, rec_chi_nblk, rec_stat_nblk;
    long long rec_step;
    unsigned long long rec_base;            // rec_ticket value the first block sees
    unsigned long long *rec_ticket;
    const double *rec_chi, *rec_stat;
    void *ring, *last;                      // m2m_record
    unsigned *cell_cache;                   // [n] packed cells of the last scatter
    int cache_read, cache_write;
    int *cell_ids;                          // [n]
    void *cell_acc;                         // [ncells] int64 fixed point or double (global atomics)
    unsigned *cell_cnt;                     // [ncells]
    int *err;
};

// Constants in the state precision: floats are rounded once on the host
// (the FP64 pipe also executes the double->float conversion).
__device__ __forceinline__ float kc(double, float f, float *) { return f; }
__device__ __forceinline__ double kc(double d, float, double *) { return d; }
#define KC(R, d, f) kc((d), (f), (R *)nullptr)

// Sign/finiteness tests of a double with integer instructions.
__device__ __forceinline__ bool d_pos(double d) {          // d > 0 (NaN false)
    long long b = __double_as_longlong(d);
    return b > 0 && b < 0x7ff0000000000001ll;
}
__device__ __forceinline__ bool d_bad(double d) {          // d < 0, NaN or +-inf
    long long b = __double_as_longlong(d);
    return b < 0 || (b & 0x7ff0000000000000ll) == 0x7ff0000000000000ll;
}

// The element at byte offset off of an array.
template <class T> __device__ __forceinline__ T *at(T *p, size_t off) { return (T *)((char *)p + off); }
template <class T> __device__ __forceinline__ const T *at(const T *p, size_t off) {
    return (const T *)((const char *)p + off);
}

// round-to-nearest integer of a float in [-2^22, 2^22] without F2I
__device__ __forceinline__ int rint_small(float x) {
    return __float_as_int(x + 12582912.0f) - 0x4B400000;
}

// ------------------------------------------------------------ TMA / mbarrier
// One-dimensional bulk copies global -> shared completing on an mbarrier
// (each warp stages its next 32-particle chunk while it computes the
// current one).  Waits are bounded: a wait that runs out returns false and
// the kernel reports M2M_ERR_TIMEOUT instead of spinning forever.
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
constexpr int MBAR_MAX_TRIES = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    for (int it = 0; it < MBAR_MAX_TRIES; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------ dependent launch
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start before the preceding kernel of its stream has
// finished; griddep_wait() returns once that kernel has completed and its
// memory is visible, so everything a kernel reads that the preceding one may
// write comes after it.  griddep_launch() lets the next kernel start early.
// Both are no-ops for kernels launched the ordinary way.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------ conversions
// Non-negative double -> float by truncation with integer instructions
// only (no FP64-pipe fallback): below the float range -> 0, above -> inf.
__device__ __forceinline__ float d2f_fast(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const int e = (int)(hi >> 20) - 896;                     // float biased exponent
    unsigned r = ((unsigned)e << 23) | (__funnelshift_l(lo, hi, 3) & 0x7fffffu);
    r = e <= 0 ? 0u : r;
    r = e >= 255 ? 0x7f800000u : r;
    return __uint_as_float(r);
}

// Float -> double with integer instructions; zero and subnormals -> 0.
__device__ __forceinline__ double f2d_fast(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xffu;
    unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    unsigned lo = b << 29;
    hi = ex == 0u ? (b & 0x80000000u) : hi;
    lo = ex == 0u ? 0u : lo;
    return __hiloint2double((int)hi, (int)lo);
}

// FP32C weights.  A double weight in the normal float range [2^-126, 2^128),
// the case the per-particle float arithmetic handles on its fast path, is
// recognised from its high word alone (negative values, zero, NaN and
// infinities fall outside), and its float value truncated toward zero (the
// d2f_fast result in this range) is the rebiased exponent and the top 23
// mantissa bits: one subtraction and one funnel shift.
__device__ __forceinline__ bool w_normal(unsigned hi) { return hi - 0x38100000u < 0x0FE00000u; }
__device__ __forceinline__ float w_to_float(unsigned hi, unsigned lo) {
    return __uint_as_float(__funnelshift_l(lo, hi - 0x38000000u, 3));
}

// Base-2 logarithm and exponential of the special-function unit with
// subnormal arguments and results flushed to zero (PTX lg2/ex2.approx.ftz):
// the logarithms here are of normal weights, and an exponential factor that
// underflows contributes nothing at the histogram's fixed-point resolution.
__device__ __forceinline__ float lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float LN2F = 0.693147180559945309f;      // ln 2
constexpr float LOG2EF = 1.44269504088896341f;     // log2 e
// e^x as 2^(x log2 e)
__device__ __forceinline__ float exp_ftz(float x) { return ex2_ftz(x * LOG2EF); }

// round(f * 2^sh) as a 64-bit integer from the float's bits (round half away
// from zero); sets *ovf when |f| * 2^sh >= 2^63.
__device__ __forceinline__ long long f2fixed(float f, int sh, bool &ovf) {
    unsigned b = __float_as_uint(f);
    int ex = (int)((b >> 23) & 0xffu);
    if (ex == 0) return 0;                         // zero / subnormal: below resolution
    if (ex == 255) { ovf = true; return 0; }
    unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
    int s = ex - 150 + sh;
    unsigned long long v;
    if (s >= 0) {
        if (s > 39) { ovf = true; return 0; }
        v = m << s;
    } else if (s > -25) {
        v = (m + (1ull << (-s - 1))) >> (-s);
    } else {
        v = 0;
    }
    long long r = (long long)v;
    return (b >> 31) ? -r : r;
}

// round(d * 2^sh) for a double (prior-cell sums of FP64 weights).
__device__ __forceinline__ long long d2fixed(double d, int sh, bool &ovf) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    int ex = (int)((b >> 52) & 0x7ffull);
    if (ex == 0) return 0;
    if (ex == 2047) { ovf = true; return 0; }
    unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
    int s = ex - 1075 + sh;
    unsigned long long v;
    if (s >= 0) {
        if (s > 10) { ovf = true; return 0; }
        v = m << s;
    } else if (s > -54) {
        v = (m + (1ull << (-s - 1))) >> (-s);
    } else {
        v = 0;
    }
    long long r = (long long)v;
    return (b >> 63) ? -r : r;
}

// Exact 64-bit accumulation into a shared (lo, hi) pair of u32 words with
// the fast 32-bit shared atomics: the carry out of the low word is detected
// from the returned old value and folded into the high-word increment, which
// is usually zero (small terms of either sign), so most updates cost one
// atomic.
__device__ __forceinline__ void fixed_add(unsigned *lo, unsigned *hi, int b, long long v) {
    unsigned vl = (unsigned)(unsigned long long)v;
    unsigned vh = (unsigned)((unsigned long long)v >> 32);
    unsigned old = atomicAdd(lo + b, vl);
    unsigned carry = (old + vl) < old ? 1u : 0u;
    unsigned inc = vh + carry;
    if (inc) atomicAdd(hi + b, inc);
}

// ------------------------------------------------------------ potentials
template <class R> struct Acc3 { R x, y, z; };

__device__ __forceinline__ float nfw_f(float r, const PotDev &p) {
    // M(r)/r^3, M = C [ln(1+u) - u/(1+u)], u = r/r_s
    float u = r * p.cf[2];
    float mu;
    if (u < 1e-2f) {
        mu = u * u * (0.5f - u * (0.6666667f - u * (0.75f - u * (0.8f - u * 0.8333333f))));
    } else {
        mu = log1pf(u) - u / (1.0f + u);
    }
    float r3 = r * r * r;
    return r > 0.f ? p.cf[0] * mu / r3 : 0.f;
}
__device__ __forceinline__ double nfw_f(double r, const PotDev &p) {
    double u = r * p.c[2];
    double mu;
    if (u < 1e-3) {
        mu = u * u * (0.5 - u * (2.0 / 3.0 - u * (0.75 - 0.8 * u)));
    } else {
        mu = log1p(u) - u / (1.0 + u);
    }
    double r3 = r * r * r;
    return r > 0. ? p.c[0] * mu / r3 : 0.;
}

// ------------------------------------------------------------ multipoles
// Even Legendre polynomials P_0..P_8 (as P[0..4]) and their derivatives by
// Bonnet's recurrence (l+1) P_(l+1) = (2l+1) mu P_l - l P_(l-1) and
// P'_(l+1) = P'_(l-1) + (2l+1) P_l.
template <class R>
__device__ __forceinline__ void legendre_even(R mu, R P[5], R dP[5]) {
    const R p1 = mu;
    const R p2 = (R(3) * mu * p1 - R(1)) * R(0.5);
    const R p3 = (R(5) * mu * p2 - R(2) * p1) * R(1.0 / 3.0);
    const R p4 = (R(7) * mu * p3 - R(3) * p2) * R(0.25);
    const R p5 = (R(9) * mu * p4 - R(4) * p3) * R(0.2);
    const R p6 = (R(11) * mu * p5 - R(5) * p4) * R(1.0 / 6.0);
    const R p7 = (R(13) * mu * p6 - R(6) * p5) * R(1.0 / 7.0);
    const R p8 = (R(15) * mu * p7 - R(7) * p6) * R(0.125);
    P[0] = R(1); P[1] = p2; P[2] = p4; P[3] = p6; P[4] = p8;
    dP[0] = R(0);
    dP[1] = R(3) * p1;
    dP[2] = dP[1] + R(7) * p3;
    dP[3] = dP[2] + R(11) * p5;
    dP[4] = dP[3] + R(15) * p7;
}

// F_l(r), D_l(r) from the node table: linear between nodes, the exterior law
// F_l(K-1) (r_(K-1)/r)^(l+1) beyond the last node, and inside the first
// F_l(0) (r/r_0)^l, D_l(0) (r/r_0)^max(l-1, 1).
template <class R>
__device__ __forceinline__ void sh_radial(R r, R ir, const R *T, const PotDev &p, R F[5], R D[5]) {
    const int K = p.ik;
    const R r0 = KC(R, p.c[1], p.cf[1]), rK = KC(R, p.c[2], p.cf[2]);
    if (r >= rK) {
        const R *row = T + (K - 1) * SH_ROW;
        const R q = rK * ir, q2 = q * q;
        R qq = q;
#pragma unroll
        for (int n = 0; n < 5; ++n) {
            F[n] = row[n] * qq;
            D[n] = -(R(2 * n + 1) * F[n]) * ir;
            qq = qq * q2;
        }
    } else if (r < r0) {
        const R q = r * KC(R, p.c[5], p.cf[5]), q2 = q * q;
        F[0] = T[0];
        D[0] = T[10] * q;
        R ql = q2, qd = q;
#pragma unroll
        for (int n = 1; n < 5; ++n) {
            F[n] = T[n] * ql;
            D[n] = T[10 + n] * qd;
            ql = ql * q2;
            qd = qd * q2;
        }
    } else {
        // segment guess from log2 r, then fixed by the node radii
        const float lg = fmaf(__log2f((float)r), p.cf[3], p.cf[4]) - 0.5f;
        int k = rint_small(fminf(fmaxf(lg, 0.0f), (float)(K - 2)));
        while (k > 0 && r < T[k * SH_ROW + 20]) --k;
        while (k < K - 2 && r >= T[(k + 1) * SH_ROW + 20]) ++k;
        const R *row = T + k * SH_ROW;
        const R dr = r - row[20];
#pragma unroll
        for (int n = 0; n < 5; ++n) {
            F[n] = row[n] + dr * row[5 + n];
            D[n] = row[10 + n] + dr * row[15 + n];
        }
    }
}

// a = -grad Phi, Phi = -sum_l P_l(mu) F_l(r):
// a = (sum P_l D_l) r_hat + (sum P_l' F_l) grad mu,
// grad mu = (-z x, -z y, x^2 + y^2) / r^3; nothing at r = 0.
template <class R>
__device__ __forceinline__ void sh_accel(R x, R y, R z, const R *T, const PotDev &p, Acc3<R> &g) {
    const R r2 = (x * x + y * y) + z * z;
    if (!(r2 > R(0))) return;
    const R r = sqrt(r2), ir = R(1) / r, mu = z * ir;
    R P[5], dP[5], F[5], D[5];
    legendre_even<R>(mu, P, dP);
    sh_radial<R>(r, ir, T, p, F, D);
    R gr = P[0] * D[0], gm = R(0);
#pragma unroll
    for (int n = 1; n < 5; ++n) {
        gr = gr + P[n] * D[n];
        gm = gm + dP[n] * F[n];
    }
    const R t = gr * ir, u = gm * ((ir * ir) * ir);
    const R c = t - u * z;
    g.x = g.x + x * c;
    g.y = g.y + y * c;
    g.z = g.z + (z * t + u * (x * x + y * y));
}

template <class R>
__device__ __forceinline__ R sh_phi(R x, R y, R z, const R *T, const PotDev &p) {
    const R r2 = (x * x + y * y) + z * z;
    if (!(r2 > R(0))) return -T[0];
    const R r = sqrt(r2), ir = R(1) / r, mu = z * ir;
    R P[5], dP[5], F[5], D[5];
    legendre_even<R>(mu, P, dP);
    sh_radial<R>(r, ir, T, p, F, D);
    R s = F[0];
#pragma unroll
    for (int n = 1; n < 5; ++n) s = s + P[n] * F[n];
    return -s;
}

// ------------------------------------------------- expansions with m != 0
// Two expansions of the weighted particles in real spherical harmonics
// beyond the axisymmetric one, each a fixed list of terms t = (l, m):
//  * triaxial (potential kind 5): the terms a set mirror-symmetric about the
//    three coordinate planes can have, even l <= 8 and even m >= 0 (cosine
//    harmonics), 15 terms (0,0) (2,0) (2,2) (4,0) .. (8,8);
//  * full (kind 6): every term up to l = 4, t = l^2 + l + m for m = -l..l,
//    25 terms (cosine harmonics for m >= 0, sine harmonics for m < 0).
// With n = x/r, mu = n_z and u = n_x + i n_y,
//   Y_lm = c_l|m| Q_l^|m|(mu) C_m,  C_m = Re u^m (m >= 0), Im u^|m| (m < 0),
//   Q_l^m = d^m P_l / dmu^m,  c_l0 = N_l0, c_lm = sqrt(2) N_lm,
//   N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
// regular on the z axis.  Node tables hold, per radial node, NT values of
//   F_t(r_k) = 4 pi/(2l+1) [A_t(r_k)/r_k^(l+1) + B_t(r_k) r_k^l],
// then their slopes to node k+1, D_t = dF_t/dr, the slopes of D, and r_k
// (4 NT + 1 values); Phi = -sum Y_t F_t(r) and, with grad C_m = |m| G_m / r,
// G_m = (Re u^(m-1), -Im u^(m-1), 0) for m > 0 and (Im u^(|m|-1),
// Re u^(|m|-1), 0) for m < 0,
//   a = sum_t [D_t Y_t n + F_t c (Q_l^(|m|+1) C (e_z - mu n)
//                                + |m| Q_l^|m| (G_m - C n)) / r].
// The terms are generated one at a time (m outer, l inner, the Q_l^m and
// Q_l^(m+1) recurrences in l carried along), so that no per-term arrays are
// live: the particle pass runs it at 64 registers a thread.
struct TriBasis {
    static constexpr int NT = 15, ROW = 4 * NT + 1, LMAX = 8, MSTEP = 2, LSTEP = 2;
    // slot of l in the radial power tables: l = 0, 2, .., 8 -> 0..4
    __host__ __device__ static constexpr int slot(int l) { return l / 2; }
    __host__ __device__ static constexpr int l_of(int t) { return t < 1 ? 0 : t < 3 ? 2 : t < 6 ? 4 : t < 10 ? 6 : 8; }
    __host__ __device__ static constexpr int t_of(int l, int m) { return (l / 2) * (l / 2 + 1) / 2 + m / 2; }
    static constexpr bool SINES = false;
};
struct FullBasis {
    static constexpr int NT = 25, ROW = 4 * NT + 1, LMAX = 4, MSTEP = 1, LSTEP = 1;
    __host__ __device__ static constexpr int slot(int l) { return l; }
    __host__ __device__ static constexpr int l_of(int t) { return t < 1 ? 0 : t < 4 ? 1 : t < 9 ? 2 : t < 16 ? 3 : 4; }
    __host__ __device__ static constexpr int t_of(int l, int m) { return l * l + l + m; }
    static constexpr bool SINES = true;
};
// backward names of the triaxial table geometry
constexpr int TRI_NT = TriBasis::NT;
constexpr int TRI_ROW = TriBasis::ROW;
constexpr int FULL_ROW = FullBasis::ROW;

// c_lm for l <= 8, 0 <= m <= l (m even or l <= 4 as the bases need)
__host__ __device__ constexpr double harm_c(int l, int m) {
    return l == 0 ? 0.28209479177387814
         : l == 1 ? (m == 0 ? 0.4886025119029199 : 0.48860251190292)
         : l == 2 ? (m == 0 ? 0.6307831305050401 : m == 1 ? 0.36418281019735976 : 0.18209140509867988)
         : l == 3 ? (m == 0 ? 0.7463526651802308 : m == 1 ? 0.3046971996429772 : m == 2 ? 0.09635371475468515
                                                                                 : 0.03933623932844291)
         : l == 4 ? (m == 0 ? 0.8462843753216345 : m == 1 ? 0.2676186174229157 : m == 2 ? 0.063078313050504
                     : m == 3 ? 0.016858388283618388 : 0.005960340337611203)
         : l == 6 ? (m == 0 ? 1.0171072362820548 : m == 2 ? 0.03509353369580661 : m == 4 ? 0.0010678622237644956
                                                                                 : 6.57223766418388e-05)
         : (m == 0 ? 1.1631066229203195 : m == 2 ? 0.023169638523677944 : m == 4 ? 0.00036818972564450655
            : m == 6 ? 7.878532816214047e-06 : 3.596041786237614e-07);
}

// Calls f(t, l, m, c, Q_l^|m|, Q_l^(|m|+1), C, Gx, Gy) for every term of
// basis B: m = 0, MSTEP, .. LMAX outer, l = m, m + LSTEP, .. LMAX inner (the
// sine term of (l, m) right after the cosine one).  Q_l^m by Q_m^m =
// (2m-1)!!, Q_(m+1)^m = (2m+1) mu Q_m^m, (l-m) Q_l^m = (2l-1) mu Q_(l-1)^m -
// (l+m-1) Q_(l-2)^m.
template <class B, class R, class Fn>
__device__ __forceinline__ void ex_terms(R mu, R nx, R ny, Fn &&f) {
    R re = R(1), im = R(0), rp = R(0), ip = R(0);    // u^m, u^(m-1)
#pragma unroll
    for (int m = 0; m <= B::LMAX; m += B::MSTEP) {
        double dfm = 1.0;                              // (2m-1)!!
        for (int k = 1; k <= m; ++k) dfm *= 2 * k - 1;
        R a1 = R(dfm), a2 = R(0);                      // Q_l^m, Q_(l-1)^m at l = m
        R b1 = R(0), b2 = R(0);                        // Q_l^(m+1), Q_(l-1)^(m+1) at l = m
#pragma unroll
        for (int l = m; l <= B::LMAX; ++l) {
            if ((l - m) % B::LSTEP == 0 || B::LSTEP == 1) {
                if (B::LSTEP == 1 || (l & 1) == 0) {
                    const R c = R(harm_c(l, m));
                    f(B::t_of(l, m), l, m, c, a1, b1, re, rp, -ip);
                    if (B::SINES && m > 0) f(B::t_of(l, -m), l, m, c, a1, b1, im, ip, rp);
                }
            }
            if (l == B::LMAX) break;
            R an, bn;
            if (l == m) an = R(2 * m + 1) * mu * a1;
            else an = (R(2 * l + 1) * mu * a1 - R(l + m) * a2) * R(1.0 / (l + 1 - m));
            if (l == m) bn = R(dfm * (2 * m + 1));     // Q_(m+1)^(m+1) = (2m+1)!!
            else if (l == m + 1) bn = R(2 * m + 3) * mu * b1;
            else bn = (R(2 * l + 1) * mu * b1 - R(l + m + 1) * b2) * R(1.0 / (l - m));
            a2 = a1; a1 = an; b2 = b1; b1 = bn;
        }
        // u^m -> u^(m + MSTEP), keeping u^(m + MSTEP - 1)
#pragma unroll
        for (int k = 0; k < B::MSTEP; ++k) {
            rp = re; ip = im;
            re = rp * nx - ip * ny;
            im = rp * ny + ip * nx;
        }
    }
}

// Radial factors of a point: F_t(r) = T[t] fa_slot + dr T[NT+t] and
// D_t(r) = T[2NT+t] da_slot + dr T[3NT+t] + (l+1) dbs F_t(r) from one table
// row: linear between nodes (fa = da = 1, dbs = 0); beyond the last node
// F(K-1) (r_(K-1)/r)^(l+1) and D = -(l+1) F/r (dr = 0, da = 0, dbs = -1/r);
// inside the first F(0) (r/r_0)^l and D(0) (r/r_0)^max(l-1, 1) (dr = 0).
template <class R> struct ExRad {
    const R *row;
    R dr, dbs, fa[5], da[5];
};

template <class B, class R>
__device__ __forceinline__ void ex_rad(R r, R ir, const R *T, const PotDev &p, ExRad<R> &g) {
    constexpr int NT = B::NT, ROW = B::ROW, S = B::LSTEP;
    const int K = p.ik;
    const R r0 = KC(R, p.c[1], p.cf[1]), rK = KC(R, p.c[2], p.cf[2]);
    g.dbs = R(0);
    g.dr = R(0);
    if (r >= rK) {
        g.row = T + (K - 1) * ROW;
        const R q = rK * ir, qs = S == 2 ? q * q : q;
        g.fa[0] = q;
#pragma unroll
        for (int n = 1; n < 5; ++n) g.fa[n] = g.fa[n - 1] * qs;
#pragma unroll
        for (int n = 0; n < 5; ++n) g.da[n] = R(0);
        g.dbs = -ir;
    } else if (r < r0) {
        g.row = T;
        const R q = r * KC(R, p.c[5], p.cf[5]), qs = S == 2 ? q * q : q;
        g.fa[0] = R(1);
#pragma unroll
        for (int n = 1; n < 5; ++n) g.fa[n] = g.fa[n - 1] * qs;
        // (r/r_0)^max(l-1, 1): q for l <= 2, then q^(l-1)
        g.da[0] = q;
#pragma unroll
        for (int n = 1; n < 5; ++n) {
            const int l = n * S;
            g.da[n] = l <= 2 ? q : g.da[n - 1] * qs;
        }
    } else {
        const float lg = fmaf(__log2f((float)r), p.cf[3], p.cf[4]) - 0.5f;
        int k = rint_small(fminf(fmaxf(lg, 0.0f), (float)(K - 2)));
        while (k > 0 && r < T[k * ROW + 4 * NT]) --k;
        while (k < K - 2 && r >= T[(k + 1) * ROW + 4 * NT]) ++k;
        g.row = T + k * ROW;
        g.dr = r - g.row[4 * NT];
#pragma unroll
        for (int n = 0; n < 5; ++n) { g.fa[n] = R(1); g.da[n] = R(1); }
    }
}

template <class B, class R>
__device__ __forceinline__ R ex_F(const ExRad<R> &g, int t, int l) {
    return g.row[t] * g.fa[B::slot(l)] + g.dr * g.row[B::NT + t];
}

template <class B, class R>
__device__ __forceinline__ void ex_accel(R x, R y, R z, const R *T, const PotDev &p, Acc3<R> &g) {
    const R r2 = (x * x + y * y) + z * z;
    if (!(r2 > R(0))) return;
    const R r = sqrt(r2), ir = R(1) / r;
    const R nx = x * ir, ny = y * ir, mu = z * ir;
    ExRad<R> rd;
    ex_rad<B, R>(r, ir, T, p, rd);
    R ar = R(0), az = R(0), ax = R(0), ay = R(0);   // along n, e_z, and G (the last two / r)
    ex_terms<B, R>(mu, nx, ny, [&](int t, int l, int m, R c, R q0, R q1, R C, R gx, R gy) {
        const R F = ex_F<B, R>(rd, t, l);
        const R D = rd.row[2 * B::NT + t] * rd.da[B::slot(l)] + rd.dr * rd.row[3 * B::NT + t] +
                    R(l + 1) * rd.dbs * F;
        const R cq0C = c * q0 * C, Fc = F * c;
        // D Y n + F c [q1 C (e_z - mu n) - m q0 C n + m q0 G] / r
        ar = ar + (D * cq0C - (Fc * q1 * C * mu + F * R(m) * cq0C) * ir);
        az = az + Fc * q1 * C;
        if (m > 0) {
            const R s = Fc * R(m) * q0;
            ax = ax + s * gx;
            ay = ay + s * gy;
        }
    });
    g.x = g.x + (ar * nx + ax * ir);
    g.y = g.y + (ar * ny + ay * ir);
    g.z = g.z + (ar * mu + az * ir);
}

template <class B, class R>
__device__ __forceinline__ R ex_phi(R x, R y, R z, const R *T, const PotDev &p) {
    const R r2 = (x * x + y * y) + z * z;
    const R r = sqrt(r2);
    const R ir = r2 > R(0) ? R(1) / r : R(0);
    const R nx = x * ir, ny = y * ir, mu = r2 > R(0) ? z * ir : R(1);
    ExRad<R> rd;
    ex_rad<B, R>(r, ir, T, p, rd);
    R s = R(0);
    ex_terms<B, R>(mu, nx, ny, [&](int t, int l, int m, R c, R q0, R q1, R C, R gx, R gy) {
        s = s + c * q0 * C * ex_F<B, R>(rd, t, l);
    });
    return -s;
}

template <class R>
__device__ __forceinline__ void tri_accel(R x, R y, R z, const R *T, const PotDev &p, Acc3<R> &g) {
    ex_accel<TriBasis, R>(x, y, z, T, p, g);
}
template <class R>
__device__ __forceinline__ R tri_phi(R x, R y, R z, const R *T, const PotDev &p) {
    return ex_phi<TriBasis, R>(x, y, z, T, p);
}
template <class R>
__device__ __forceinline__ void full_accel(R x, R y, R z, const R *T, const PotDev &p, Acc3<R> &g) {
    ex_accel<FullBasis, R>(x, y, z, T, p, g);
}
template <class R>
__device__ __forceinline__ R full_phi(R x, R y, R z, const R *T, const PotDev &p) {
    return ex_phi<FullBasis, R>(x, y, z, T, p);
}

// Potential signatures compiled into the steady-state kernels (the generic
// form walks the component list at run time):
enum { PK_ANY = 0, PK_HERNQUIST = 1, PK_LOG = 3, PK_SH = 4, PK_HERNQUIST_NFW = 5, PK_SH_TRI = 6, PK_SH_FULL = 7 };

template <class R>
__device__ __forceinline__ void acc_hernquist(R x, R y, R z, const PotDev &p, Acc3<R> &g) {
    R GM = KC(R, p.c[0], p.cf[0]), aa = KC(R, p.c[1], p.cf[1]);
    R r2 = (x * x + y * y) + z * z;
    R r = sqrt(r2);
    R s = r + aa;
    R f = r2 > R(0) ? GM / ((r * s) * s) : R(0);
    g.x = g.x + (-(f * x));
    g.y = g.y + (-(f * y));
    g.z = g.z + (-(f * z));
}
template <class R>
__device__ __forceinline__ void acc_log(R x, R y, R z, const PotDev &p, Acc3<R> &g) {
    R Rc2 = KC(R, p.c[0], p.cf[0]), iq2 = KC(R, p.c[1], p.cf[1]), v0sq = KC(R, p.c[2], p.cf[2]);
    R R2 = x * x + y * y;
    R D = (Rc2 + R2) + (z * z) * iq2;
    R f = v0sq / D;
    g.x = g.x + (-(f * x));
    g.y = g.y + (-(f * y));
    g.z = g.z + (-((f * iq2) * z));
}
template <class R>
__device__ __forceinline__ void acc_nfw(R x, R y, R z, const PotDev &p, Acc3<R> &g) {
    R r2 = (x * x + y * y) + z * z;
    R f = nfw_f(sqrt(r2), p);
    g.x = g.x + (-(f * x));
    g.y = g.y + (-(f * y));
    g.z = g.z + (-(f * z));
}

// A single component's acceleration itself (the sum over components below
// starts from zero; 0 + v equals v except for the sign of a zero, which no
// later comparison sees).
template <class R>
__device__ __forceinline__ Acc3<R> acc1_hernquist(R x, R y, R z, const PotDev &p) {
    R GM = KC(R, p.c[0], p.cf[0]), aa = KC(R, p.c[1], p.cf[1]);
    R r2 = (x * x + y * y) + z * z;
    R r = sqrt(r2);
    R s = r + aa;
    R f = r2 > R(0) ? GM / ((r * s) * s) : R(0);
    return Acc3<R>{-(f * x), -(f * y), -(f * z)};
}
template <class R>
__device__ __forceinline__ Acc3<R> acc1_log(R x, R y, R z, const PotDev &p) {
    R Rc2 = KC(R, p.c[0], p.cf[0]), iq2 = KC(R, p.c[1], p.cf[1]), v0sq = KC(R, p.c[2], p.cf[2]);
    R R2 = x * x + y * y;
    R D = (Rc2 + R2) + (z * z) * iq2;
    R f = v0sq / D;
    return Acc3<R>{-(f * x), -(f * y), -((f * iq2) * z)};
}

template <class R, int PK = PK_ANY>
__device__ __forceinline__ Acc3<R> accel(R x, R y, R z, const PassArgs &a, const R *sh = nullptr) {
    Acc3<R> g{R(0), R(0), R(0)};
    if constexpr (PK == PK_HERNQUIST) {
        return acc1_hernquist<R>(x, y, z, a.pot[0]);
    } else if constexpr (PK == PK_LOG) {
        return acc1_log<R>(x, y, z, a.pot[0]);
    } else if constexpr (PK == PK_SH) {
        sh_accel<R>(x, y, z, sh, a.pot[0], g);
        return g;
    } else if constexpr (PK == PK_SH_TRI) {
        tri_accel<R>(x, y, z, sh, a.pot[0], g);
        return g;
    } else if constexpr (PK == PK_SH_FULL) {
        full_accel<R>(x, y, z, sh, a.pot[0], g);
        return g;
    } else if constexpr (PK == PK_HERNQUIST_NFW) {
        acc_hernquist<R>(x, y, z, a.pot[0], g);
        acc_nfw<R>(x, y, z, a.pot[1], g);
        return g;
    }
    for (int k = 0; k < a.npot; ++k) {
        const PotDev &p = a.pot[k];
        if (p.kind == 1) {            // Hernquist
            acc_hernquist<R>(x, y, z, p, g);
        } else if (p.kind == 3) {     // flattened logarithmic
            acc_log<R>(x, y, z, p, g);
        } else if (p.kind == 2) {     // NFW
            acc_nfw<R>(x, y, z, p, g);
        } else if (p.kind == 4) {     // spherical harmonics of the particles
            sh_accel<R>(x, y, z, sh, p, g);
        } else if (p.kind == 5) {     // the triaxial expansion of the particles
            tri_accel<R>(x, y, z, sh, p, g);
        } else if (p.kind == 6) {     // the full expansion (l <= 4) of the particles
            full_accel<R>(x, y, z, sh, p, g);
        }
    }
    return g;
}

// ln x in float arithmetic with a fixed operation order, so that the
// energy of the prior cells (and each particle's cell) does not depend on a
// library's rounding of the logarithm.  From ln m = 2 atanh(s) = 2 (s +
// s^3/3 + ... + s^9/9 + ...), s = (m - 1)/(m + 1), after x = 2^k m with m in
// [sqrt(1/2), sqrt(2)] (|s| <= 0.1716: truncation error below 1e-9
// relative): every product and sum rounded separately, the coefficients
// 2/(2j+1) rounded to float, ln 2 = LN2_HI + LN2_LO with LN2_HI =
// 0x3f317200 (k LN2_HI exact).  Subnormal x scaled by 2^24 first; 0 ->
// -inf, negative or NaN -> NaN, +inf -> +inf.
__device__ __forceinline__ float log_det(float x) {
    if (!(x > 0.f) || x == INFINITY) return x == 0.f ? -INFINITY : (x == INFINITY ? INFINITY : __int_as_float(0x7fc00000));
    int ks = 0;
    if (x < 1.17549435e-38f) { x = __fmul_rn(x, 16777216.0f); ks = -24; }
    const unsigned b = __float_as_uint(x);
    int k = (int)(b >> 23) - 127 + ks;
    unsigned mb = (b & 0x007FFFFFu) | 0x3F800000u;
    if (mb > 0x3FB504F3u) { mb -= 0x00800000u; k += 1; }
    const float m = __uint_as_float(mb);
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(s, s);
    // 2/9, 2/7, 2/5, 2/3 and 2 as the floats nearest their double values
    float p = __uint_as_float(0x3E638E39u);
    p = __fadd_rn(__fmul_rn(p, z), __uint_as_float(0x3E924925u));
    p = __fadd_rn(__fmul_rn(p, z), __uint_as_float(0x3ECCCCCDu));
    p = __fadd_rn(__fmul_rn(p, z), __uint_as_float(0x3F2AAAABu));
    p = __fadd_rn(__fmul_rn(p, z), 2.0f);
    const float lm = __fmul_rn(s, p);
    const float kf = (float)k;
    const float LN2_HI = __uint_as_float(0x3F317200u), LN2_LO = __uint_as_float(0x35BFBE8Eu);
    return __fadd_rn(__fmul_rn(kf, LN2_HI), __fadd_rn(__fmul_rn(kf, LN2_LO), lm));
}
// The same in double: terms to s^21 (truncation below 1e-17 relative),
// LN2_HI = ln 2 with its low 32 mantissa bits cleared, LN2_LO the rest of
// the double ln 2; subnormal x scaled by 2^54 first.
__device__ __forceinline__ double log_det(double x) {
    if (!(x > 0.0) || x == (double)INFINITY)
        return x == 0.0 ? -(double)INFINITY : (x == (double)INFINITY ? (double)INFINITY : __longlong_as_double(0x7ff8000000000000ll));
    int ks = 0;
    if (x < 2.2250738585072014e-308) { x = __dmul_rn(x, 18014398509481984.0); ks = -54; }
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int k = (int)(b >> 52) - 1023 + ks;
    unsigned long long mb = (b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    if (mb > 0x3FF6A09E667F3BCCull) { mb -= 0x0010000000000000ull; k += 1; }
    const double m = __longlong_as_double((long long)mb);
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    // 2/21, 2/19, ..., 2/3, 2 as the doubles nearest them
    const unsigned long long cb[11] = {0x3FB8618618618618ull, 0x3FBAF286BCA1AF28ull, 0x3FBE1E1E1E1E1E1Eull,
                                       0x3FC1111111111111ull, 0x3FC3B13B13B13B14ull, 0x3FC745D1745D1746ull,
                                       0x3FCC71C71C71C71Cull, 0x3FD2492492492492ull, 0x3FD999999999999Aull,
                                       0x3FE5555555555555ull, 0x4000000000000000ull};
    double p = __longlong_as_double((long long)cb[0]);
#pragma unroll
    for (int j = 1; j < 11; ++j) p = __dadd_rn(__dmul_rn(p, z), __longlong_as_double((long long)cb[j]));
    const double lm = __dmul_rn(s, p);
    const double kf = (double)k;
    const double LN2_HI = __longlong_as_double(0x3FE62E4200000000ll), LN2_LO = __longlong_as_double(0x3E9FDF473DE00000ll);
    return __dadd_rn(__dmul_rn(kf, LN2_HI), __dadd_rn(__dmul_rn(kf, LN2_LO), lm));
}
__device__ __forceinline__ float plog(float v) { return log_det(v); }
__device__ __forceinline__ double plog(double v) { return log_det(v); }

// One component's term of Phi (kinds 1 Hernquist, 3 flattened log, 2 NFW,
// 4 spherical harmonics); the sum is taken in component order from 0.
template <class R>
__device__ __forceinline__ R phi_term(int kind, R x, R y, R z, const PotDev &p, const R *sh) {
    if (kind == 1) {
        R GM = KC(R, p.c[0], p.cf[0]), aa = KC(R, p.c[1], p.cf[1]);
        R r2 = (x * x + y * y) + z * z;
        return -(GM / (sqrt(r2) + aa));
    } else if (kind == 3) {
        R Rc2 = KC(R, p.c[0], p.cf[0]), iq2 = KC(R, p.c[1], p.cf[1]), hv = KC(R, p.c[3], p.cf[3]);
        R R2 = x * x + y * y;
        R D = (Rc2 + R2) + (z * z) * iq2;
        return hv * plog(D);
    } else if (kind == 2) {
        // Phi = -C ln(1+u)/r, C = 4 pi rho_s r_s^3, evaluated in double
        // and rounded once; the r -> 0 limit is -C / r_s
        double xd = x, yd = y, zd = z;
        double r = sqrt(xd * xd + yd * yd + zd * zd);
        double u = r * p.c[2];
        double v = r > 0 ? -p.c[0] * log1p(u) / r : -p.c[0] * p.c[2];
        return (R)v;
    } else if (kind == 4) {
        return sh_phi<R>(x, y, z, sh, p);
    } else if (kind == 5) {
        return tri_phi<R>(x, y, z, sh, p);
    } else if (kind == 6) {
        return full_phi<R>(x, y, z, sh, p);
    }
    return R(0);
}

// Phi at (x, y, z): the compiled signatures take the same terms in the
// same order as the run-time walk of the component list.
template <class R, int PK = PK_ANY>
__device__ __forceinline__ R potential(R x, R y, R z, const PassArgs &a, const R *sh = nullptr) {
    R phi = R(0);
    if constexpr (PK == PK_HERNQUIST) {
        return phi + phi_term<R>(1, x, y, z, a.pot[0], sh);
    } else if constexpr (PK == PK_LOG) {
        return phi + phi_term<R>(3, x, y, z, a.pot[0], sh);
    } else if constexpr (PK == PK_SH) {
        return phi + phi_term<R>(4, x, y, z, a.pot[0], sh);
    } else if constexpr (PK == PK_SH_TRI) {
        return phi + phi_term<R>(5, x, y, z, a.pot[0], sh);
    } else if constexpr (PK == PK_SH_FULL) {
        return phi + phi_term<R>(6, x, y, z, a.pot[0], sh);
    } else if constexpr (PK == PK_HERNQUIST_NFW) {
        phi = phi + phi_term<R>(1, x, y, z, a.pot[0], sh);
        return phi + phi_term<R>(2, x, y, z, a.pot[1], sh);
    }
    for (int k = 0; k < a.npot; ++k) phi = phi + phi_term<R>(a.pot[k].kind, x, y, z, a.pot[k], sh);
    return phi;
}

// With an expansion potential the force at the new positions is kept
// (a.facc, [3][n] in the state precision) and, while neither the positions
// nor the node table have changed since (a.facc_read), taken instead of a
// second evaluation at the start of the next push: the same function of the
// same arguments, so the same bits.
template <class R, int PK = PK_ANY>
__device__ __forceinline__ void kdk(R &x, R &y, R &z, R &vx, R &vy, R &vz, const PassArgs &a,
                                    const R *sh = nullptr, long long i = 0) {
    R h = KC(R, a.hdt, a.f_hdt), d = KC(R, a.dt, a.f_dt);
    constexpr bool CACHE = PK == PK_ANY || PK == PK_SH || PK == PK_SH_TRI || PK == PK_SH_FULL;
    R *fc = CACHE ? (R *)a.facc : nullptr;
    Acc3<R> g;
    if (CACHE && fc && a.facc_read) {
        g.x = fc[i];
        g.y = fc[a.n + i];
        g.z = fc[2 * a.n + i];
    } else {
        g = accel<R, PK>(x, y, z, a, sh);
    }
    vx = vx + h * g.x;
    vy = vy + h * g.y;
    vz = vz + h * g.z;
    x = x + d * vx;
    y = y + d * vy;
    z = z + d * vz;
    g = accel<R, PK>(x, y, z, a, sh);
    if (CACHE && fc) {
        fc[i] = g.x;
        fc[a.n + i] = g.y;
        fc[2 * a.n + i] = g.z;
    }
    vx = vx + h * g.x;
    vy = vy + h * g.y;
    vz = vz + h * g.z;
}

// ------------------------------------------------------------ bin search
// Cell j with e[j] <= v < e[j+1], j in [0, nb), else -1.  The guess only
// shortens the search; the result is fixed by the comparisons.
template <class R>
__device__ __forceinline__ int find_bin(R v, const R *e, int nb, int mode, float ga, float gb) {
    if (!(v >= e[0] && v < e[nb])) return -1;
    int j;
    if (mode == G_BIS) {
        int lo = 0, hi = nb;              // e[lo] <= v < e[hi]
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (v >= e[mid]) lo = mid; else hi = mid;
        }
        return lo;
    }
    float fv = (float)v;
    float gg = (mode == G_LOG) ? fmaf(ga, __log2f(fv), gb) : fmaf(ga, fv, gb);
    j = (gg >= 0.f) ? (int)gg : 0;
    j = j < nb - 1 ? j : nb - 1;
    while (v < e[j]) --j;                 // terminates: v >= e[0]
    while (v >= e[j + 1]) ++j;            // terminates: v < e[nb]
    return j;
}

// Number of interior edges e[1..nc-1] with e[k] <= v (NaN -> 0), in [0, nc-1];
// e[] is indexed 0..nc with e[0], e[nc] unused.
template <class R>
__device__ __forceinline__ int count_le(R v, const R *e, int nc, float ga, float gb) {
    if (!(v == v)) return 0;
    float gg = fmaf(ga, (float)v, gb);
    int j = (gg >= 0.f) ? (gg < (float)nc ? (int)gg : nc - 1) : 0;
    if (j > nc - 1) j = nc - 1;
    while (j > 0 && !(e[j] <= v)) --j;
    while (j < nc - 1 && e[j + 1] <= v) ++j;
    return j;
}

// ------------------------------------------------------------ GH kernel
// u_n(nu; s) = 2 sqrt(pi) N(nu; 0, 1+s^2) E_{N(m, t2)}[H_n], m = nu c1,
// c1 = 1/(1+s^2), t2 = s^2 c1; table per cell: V, 1/S, c1, t2, norm with
// norm = 2 sqrt(pi) / sqrt(2 pi (1+s^2)).
__device__ __forceinline__ void gh_eval(float vlos, const float *g, float u[5]) {
    const float SQ2 = 1.41421356237f, ISQ2 = 0.707106781187f, ISQ3 = 0.57735026919f,
                ISQ24 = 0.204124145232f;
    float nu = (vlos - g[0]) * g[1];
    float c1 = g[2], t2 = g[3];
    float gs = g[4] * exp_ftz(-0.5f * nu * nu * c1);
    float m = nu * c1, m2 = m * m;
    float E2 = m2 + t2;
    float E3 = m * fmaf(3.f, t2, m2);
    float E4 = fmaf(m2, m2, fmaf(6.f * m2, t2, 3.f * t2 * t2));
    u[0] = gs;
    u[1] = gs * (SQ2 * m);
    u[2] = gs * (fmaf(2.f, E2, -1.f) * ISQ2);
    u[3] = gs * (fmaf(2.f, E3, -3.f * m) * ISQ3);
    u[4] = gs * (fmaf(4.f, E4, fmaf(-12.f, E2, 3.f)) * ISQ24);
}
__device__ __forceinline__ void gh_eval(double vlos, const double *g, double u[5]) {
    const double SQ2 = 1.4142135623730951, SQ3 = 1.7320508075688772, SQ24 = 4.898979485566356;
    double nu = (vlos - g[0]) * g[1];
    double c1 = g[2], t2 = g[3];
    double gs = g[4] * exp(-0.5 * nu * nu * c1);
    double m = nu * c1, m2 = m * m;
    double E2 = m2 + t2;
    double E3 = m * m2 + 3.0 * m * t2;
    double E4 = m2 * m2 + 6.0 * m2 * t2 + 3.0 * t2 * t2;
    u[0] = gs;
    u[1] = gs * (SQ2 * m);
    u[2] = gs * ((2.0 * E2 - 1.0) / SQ2);
    u[3] = gs * ((2.0 * E3 - 3.0 * m) / SQ3);
    u[4] = gs * ((4.0 * E4 - 12.0 * E2 + 3.0) / SQ24);
}

// The per-cell record of the compiled FP32C layouts (three float4):
//   r[0] = (V, c1/S, -log2(e)/(2S), log2 norm), r[1] = (P0, P1, P2, P3),
//   r[2] = (P4, d/sqrt 2, sqrt 3 d, 12 d/sqrt 24),  d = 2 t2 - 1,
// P0..P4 the update's quartic of the step (without the norm).  With
// dv = v_los - V and m = dv c1/S (= nu c1), the Gaussian factor of every
// term is g = norm exp(-nu m/2) = 2^(dv m (-log2(e)/(2S)) + log2 norm), and
// the van der Marel & Franx moments of gh_eval become, with m2 = m^2,
//   u0 = g, u1 = g sqrt2 m, u2 = g (sqrt2 m2 + d/sqrt2),
//   u3 = g m (2/sqrt3 m2 + sqrt3 d),
//   u4 = g (4/sqrt24 m2^2 + 12 d/sqrt24 m2 + 3 d^2/sqrt24)
// (E2 = m2 + t2 etc. expanded: 2 E2 - 1 = 2 m2 + d, 2 E3 - 3 m = m (2 m2 +
// 3 d), 4 E4 - 12 E2 + 3 = 4 m2^2 + 12 d m2 + 3 d^2), the last constant
// 3 d^2/sqrt24 = (12 d/sqrt24)^2 / (2 sqrt24).
__device__ __forceinline__ void gh_record(float V, float iS, float c1, float t2, float nrm, const float P[5],
                                          float4 r[3]) {
    const float d = fmaf(2.f, t2, -1.f);
    r[0] = make_float4(V, c1 * iS, (-0.5f * 1.44269504088896341f) * iS, log2f(nrm));
    r[1] = make_float4(P[0], P[1], P[2], P[3]);
    r[2] = make_float4(P[4], d * 0.707106781187f, d * 1.73205080757f, d * 2.44948974278f);
}

// The five moments of one particle from a cell record (the arithmetic of
// the scatter's fast path, which adds each term as it is formed).
__device__ __forceinline__ void gh_eval_rec(float vlos, const float4 *r, float u[5]) {
    const float SQ2 = 1.41421356237f, K3 = 1.15470053838f, K4 = 0.816496580928f, C4 = 0.102062072616f;
    const float4 a = r[0], c = r[2];
    const float dv = vlos - a.x, m = dv * a.y, m2 = m * m;
    const float g = ex2_ftz(fmaf(dv * m, a.z, a.w));
    u[0] = g;
    u[1] = g * (SQ2 * m);
    u[2] = g * fmaf(SQ2, m2, c.y);
    u[3] = g * (m * fmaf(K3, m2, c.z));
    u[4] = g * fmaf(m2, fmaf(K4, m2, c.w), (c.w * c.w) * C4);
}

__device__ __forceinline__ float gh_exp(float x) { return exp_ftz(x); }
__device__ __forceinline__ double gh_exp(double x) { return exp(x); }

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, SC'11): the
// round multipliers and Weyl key increments of that publication.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The sky position of particle i seen through set k's PSF at positions that
// have had `epoch` pushes: one draw, two table entries, added in the state
// precision.
template <class R>
__device__ __forceinline__ void seeing(const SetDev &s, int k, long long i, long long epoch, R &X, R &Ys) {
    const uint4 u = philox4x32_10(make_uint4((unsigned)i, (unsigned)epoch, (unsigned)k,
                                             (unsigned)((unsigned long long)epoch >> 32)),
                                  make_uint2(s.psf_seed, 0u));
    const R *q = (const R *)s.psf;
    X = X + __ldg(q + (u.x >> s.psf_shift));
    Ys = Ys + __ldg(q + (u.y >> s.psf_shift));
}

// Cell of particle in set s (-1 = none).  X = x, Ys = z*sin - y*cos.
template <class R>
__device__ __forceinline__ int set_cell(const SetDev &s, const R *edges, R x, R y, R z, R X, R Ys) {
    if (s.geom == 1) {
        R r2 = (x * x + y * y) + z * z;
        return find_bin<R>(r2, edges + s.ex_off, s.nx, s.gx_mode, s.gx_a, s.gx_b);
    } else if (s.geom == 2) {
        R R2 = X * X + Ys * Ys;
        return find_bin<R>(R2, edges + s.ex_off, s.nx, s.gx_mode, s.gx_a, s.gx_b);
    } else {
        int ix = find_bin<R>(X, edges + s.ex_off, s.nx, s.gx_mode, s.gx_a, s.gx_b);
        if (ix < 0) return -1;
        int iy = find_bin<R>(Ys, edges + s.ey_off, s.ny, s.gy_mode, s.gy_a, s.gy_b);
        if (iy < 0) return -1;
        // grid: the pixel is the cell; lookup table: the pixel's aperture
        return s.geom == 4 ? __ldg(s.lut + iy * s.nx + ix) : iy * s.nx + ix;
    }
}


// Branch-free cell lookup for edge tables whose index guess (linear or
// log2, fitted on the host) is within one cell of the true cell everywhere
// in range: one correction step on each side, decided by the two edges of
// the guessed cell.  Same membership as find_bin.
// Both edges of cell k as one shared-memory load: (e[k], e[k+1]).
template <class R> struct EdgePair;
template <> struct EdgePair<float> { using T = float2; };
template <> struct EdgePair<double> { using T = double2; };
template <class R> using Pair = typename EdgePair<R>::T;

template <class R, int MODE>
__device__ __forceinline__ int find_fast(R v, const Pair<R> *e, int nb, float ga, float gb, float top) {
    const float fv = (float)v;
    const float t = MODE == G_LOG ? __log2f(fv) : fv;
    // nearest integer to (guess - 1/2), clamped to the table: within one cell
    // of the true cell for any v in range, which the two edge tests pin down;
    // a v outside the table (or NaN) ends outside [0, nb)
    const float gf = fminf(fmaxf(fmaf(ga, t, gb) - 0.5f, 0.0f), top);
    int g = rint_small(gf);
    const Pair<R> ed = e[g];
    g += (v >= ed.y ? 1 : 0) - (v < ed.x ? 1 : 0);
    return ((unsigned)g < (unsigned)nb && v == v) ? g : -1;
}

// Cell of a particle in a set of compile-time geometry G whose edge tables
// are uniform in value (G_LIN: grids, lookup tables) or in log (G_LOG:
// shells, annuli).
template <class R, int G>
__device__ __forceinline__ int cell_t(const SetDev &s, const Pair<R> *edges, R x, R y, R z, R X, R Ys) {
    if constexpr (G == 1) {
        R r2 = (x * x + y * y) + z * z;
        return find_fast<R, G_LOG>(r2, edges + s.ex_off, s.nx, s.gx_a, s.gx_b, s.gx_top);
    } else if constexpr (G == 2) {
        R R2 = X * X + Ys * Ys;
        return find_fast<R, G_LOG>(R2, edges + s.ex_off, s.nx, s.gx_a, s.gx_b, s.gx_top);
    } else {
        int ix = find_fast<R, G_LIN>(X, edges + s.ex_off, s.nx, s.gx_a, s.gx_b, s.gx_top);
        int iy = find_fast<R, G_LIN>(Ys, edges + s.ey_off, s.ny, s.gy_a, s.gy_b, s.gy_top);
        if constexpr (G == 4)          // lookup table: the aperture that owns the pixel
            return (ix < 0 || iy < 0) ? -1 : __ldg(s.lut + iy * s.nx + ix);
        return (ix < 0 || iy < 0) ? -1 : iy * s.nx + ix;
    }
}

// Fixed-point histogram add of a float term v, V = round(v * 2^sh) (a
// 64-bit integer), kept as three int32 sums per bin in shared memory:
// V = A * 2^32 + B * 2^16 + L with |B| <= 2^15 and |L| <= 2^16.  Every part
// goes in with a plain reduction (no returned value, no carry), and the bin
// total is A_sum * 2^32 + B_sum * 2^16 + L_sum.  It is exact while at most
// 2^15 terms reach a bin between two flushes (the pass flushes every
// 32768 particles of a block), which keeps |B_sum|, |L_sum| < 2^31; A_sum
// stays in range for any |V| < 2^62.  A is 0 for the usual terms (|V| <
// 2^31, the fast path: V by one round-to-nearest conversion, L = V mod 2^16
// and B = V >> 16) and its reduction is skipped.  For |V| < 2^38 the split
// takes two exact float steps (1.5*2^23 "magic" rounding of V/2^16, then of
// the exact remainder V - h*2^16), larger terms take the bit-level path.
// fscale = 2^sh as a float (an exact power of two).
constexpr float FX_MAGIC = 12582912.0f;            // 1.5 * 2^23
// The common case of fx_red, for |S| = |v * 2^sh| < 2^31 (A = 0): the two
// lower parts only, no range test; the caller checks the range once for all
// of a particle's terms of one observable set.
constexpr float FX_FAST = 2147483648.0f;           // 2^31
__device__ __forceinline__ void fx_red_fast(int *Lo, int *Mid, int b, float S) {
    const int V = __float2int_rn(S);                           // round to nearest even, |S| < 2^31
    atomicAdd(Lo + b, V & 0xFFFF);
    atomicAdd(Mid + b, V >> 16);
}
// The five Gauss-Hermite terms of one particle (the arithmetic of
// gh_eval_rec), each scaled by W = w 2^sh and added to the histogram as soon
// as it is formed (|W u_n| < 2^31 is the caller's test), to keep few values
// live.
__device__ __forceinline__ void gh_red_stream(float vlos, const float4 *r, float W, int *Lo, int *Mid, int b) {
    const float SQ2 = 1.41421356237f, K3 = 1.15470053838f, K4 = 0.816496580928f, C4 = 0.102062072616f;
    const float4 a = r[0], c = r[2];
    const float dv = vlos - a.x, m = dv * a.y;
    const float Wg = W * ex2_ftz(fmaf(dv * m, a.z, a.w));
    const float m2 = m * m;
    fx_red_fast(Lo, Mid, b, Wg);
    fx_red_fast(Lo, Mid, b + 1, Wg * (SQ2 * m));
    fx_red_fast(Lo, Mid, b + 2, Wg * fmaf(SQ2, m2, c.y));
    fx_red_fast(Lo, Mid, b + 3, Wg * (m * fmaf(K3, m2, c.z)));
    fx_red_fast(Lo, Mid, b + 4, Wg * fmaf(m2, fmaf(K4, m2, c.w), (c.w * c.w) * C4));
}

__device__ __forceinline__ void fx_red(int *Lo, int *Mid, int *Hi, int b, float v, float fscale, int sh,
                                       bool &ovf) {
    const float S = v * fscale;
    int h, l;
    if (fabsf(S) < 274877906944.0f) {                          // 2^38
        const float t = fmaf(S, 1.52587890625e-05f, FX_MAGIC); // round(S / 2^16) + M
        h = __float_as_int(t) - 0x4B400000;
        const float r = fmaf(-(t - FX_MAGIC), 65536.0f, S);    // S - h * 2^16, exact
        l = __float_as_int(r + FX_MAGIC) - 0x4B400000;
        const int A = (h + 32768) >> 16;
        atomicAdd(Lo + b, l);
        atomicAdd(Mid + b, h - (A << 16));
        if (A) atomicAdd(Hi + b, A);
    } else {
        const long long q = f2fixed(v, sh, ovf);
        const long long hh = (q + 32768) >> 16;
        const long long A = (hh + 32768) >> 16;
        atomicAdd(Lo + b, (int)(q - (hh << 16)));
        atomicAdd(Mid + b, (int)(hh - (A << 16)));
        atomicAdd(Hi + b, (int)A);
    }
}

}  // namespace m2m
