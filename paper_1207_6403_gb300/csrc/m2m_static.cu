// m2m_observe_static: observables of a particle set with no device
// allocation.
//
// Some callers cannot allocate device memory at the moment they need an
// observation: code running under an external memory manager that owns
// every allocation, allocator-free real-time or embedded deployments, and
// callers that must not trigger the implicit synchronisation a
// cudaMalloc/cudaFree can cause.  For them this entry
// point runs the same scatter kernel as m2m_observe (FP32-compensated,
// exact fixed-point sums) with all of its scratch -- the integer observable
// totals, the error word and the edge and Gauss-Hermite tables -- kept in
// one file-scope device array of fixed size instead of allocated buffers.
// The caller passes the particle arrays and the output array.
//
// The array lives in every GPU that loads the library until the process
// exits (M2M_STATIC_SCRATCH_BYTES).  All calls share it: calls that overlap
// on the GPU (other streams, other host threads) race and give wrong
// results.  The totals are cleared at the start of every call.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "m2m.h"
#include "m2m_kernels.cuh"

using namespace m2m;

namespace {

// scratch layout (bytes): int64 totals | error word | edge table | GH table
constexpr size_t OFF_TOT = 0;
constexpr size_t OFF_ERR = OFF_TOT + 8ull * M2M_STATIC_MAX_OBS;
constexpr size_t OFF_EDGES = OFF_ERR + 256;
constexpr size_t OFF_GH = OFF_EDGES + 4ull * M2M_STATIC_MAX_EDGES;
constexpr size_t SCRATCH_END = OFF_GH + 4ull * 5 * M2M_STATIC_MAX_GH_CELLS;
static_assert(SCRATCH_END <= M2M_STATIC_SCRATCH_BYTES, "scratch layout exceeds the array");

}  // namespace

// The scratch itself.  Host code may not use this name as an address: it
// is only a handle for cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_m2m_static_scratch[M2M_STATIC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[MAX_DEVICES];   // device address of the array, per device
int g_nsm[MAX_DEVICES];
// Messages go where m2m_last_error(NULL) reads them.
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    note_context_free_error(buf);
    return code;
}

// Once per device, with that device current: the array's device address,
// the SM count and the kernels' shared-memory limits.
int setup_device(int dev) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev]) return M2M_OK;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_m2m_static_scratch);
    if (e != cudaSuccess || !p) return fail(M2M_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    int nsm = 0, optin = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int lay = 0; lay < 4 && e == cudaSuccess; ++lay) {
        void *f = pass_kernel_f32(1024, lay);
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, f);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    }
    if (e != cudaSuccess) return fail(M2M_ERR_CUDA, "device set-up: %s", cudaGetErrorString(e));
    g_nsm[dev] = nsm;
    g_scratch_ptr[dev] = (unsigned char *)p;
    return M2M_OK;
}

float ceil_float(double e) {
    float f = (float)e;
    if ((double)f < e) f = nextafterf(f, INFINITY);
    return f;
}

// Index guess of an edge table, as for contexts: linear or log2 when the
// fit predicts every edge within 0.01 cell, else bisection.
void guess_params(const double *e, int nb, int *mode, float *ga, float *gb) {
    double span = e[nb] - e[0];
    bool lin_ok = span > 0 && isfinite(span);
    if (lin_ok) {
        double a = nb / span, b = -e[0] * a;
        for (int k = 0; k <= nb && lin_ok; ++k)
            if (fabs(a * e[k] + b - k) > 0.01) lin_ok = false;
        if (lin_ok) { *mode = G_LIN; *ga = (float)a; *gb = (float)b; return; }
    }
    if (e[0] > 0) {
        double l0 = log2(e[0]), l1 = log2(e[nb]);
        bool ok = l1 > l0;
        double a = ok ? nb / (l1 - l0) : 0, b = -l0 * a;
        for (int k = 0; k <= nb && ok; ++k)
            if (fabs(a * log2(e[k]) + b - k) > 0.01) ok = false;
        if (ok) { *mode = G_LOG; *ga = (float)a; *gb = (float)b; return; }
    }
    *mode = G_BIS; *ga = 0.f; *gb = 0.f;
}

int layout_of(const SetDev *sets, int nsets) {
    for (int k = 0; k < nsets; ++k) {
        const SetDev &s = sets[k];
        if (s.geom == M2M_GEOM_GRID && (s.gx_mode != G_LIN || s.gy_mode != G_LIN)) return 0;
        if (s.geom != M2M_GEOM_GRID && s.gx_mode != G_LOG) return 0;
    }
    auto is = [&](int k, int g, int q) { return sets[k].geom == g && sets[k].quant == q; };
    if (nsets == 2 && is(0, M2M_GEOM_GRID, M2M_Q_MASS) && is(1, M2M_GEOM_GRID, M2M_Q_GH)) return 1;
    if (nsets == 2 && is(0, M2M_GEOM_SHELL, M2M_Q_MASS) && is(1, M2M_GEOM_ANNULUS, M2M_Q_GH)) return 2;
    if (nsets == 3 && is(0, M2M_GEOM_SHELL, M2M_Q_MASS) && is(1, M2M_GEOM_ANNULUS, M2M_Q_MASS) &&
        is(2, M2M_GEOM_ANNULUS, M2M_Q_VLOS2))
        return 3;
    return 0;
}

// y_j = total_j * q; the totals are cleared for the next call.  An overflow
// or non-finite weight found by the scatter turns every output into NaN.
__global__ void k_static_finish(unsigned long long *tot, const int *err, double *y, int nobs, double q) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nobs) return;
    const unsigned long long t = tot[j];
    tot[j] = 0ull;
    y[j] = *err ? __longlong_as_double(0x7ff8000000000000ll) : (double)(long long)t * q;
}

}  // namespace

extern "C" {

int m2m_observe_static(int64_t n, const void *x, const void *y, const void *z, const void *vx,
                       const void *vy, const void *vz, const double *w, const m2m_obs_desc *obs,
                       int32_t nsets, double incl_sin, double incl_cos, double weight_scale,
                       double *y_out, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 1 || n >= (1ll << 31)) return fail(M2M_ERR_ARG, "n=%lld out of [1, 2^31)", (long long)n);
    const void *arrs[] = {x, y, z, vx, vy, vz, w, y_out};
    for (int k = 0; k < 8; ++k)
        if (!arrs[k] || ((uintptr_t)arrs[k] & 15u))
            return fail(M2M_ERR_ARG, "array %d is NULL or not 16-byte aligned", k);
    if (nsets < 1 || nsets > MAXSETS || !obs) return fail(M2M_ERR_ARG, "nsets=%d out of [1,%d]", nsets, MAXSETS);
    if (!(weight_scale > 0) || !isfinite(weight_scale) || !isfinite(incl_sin) || !isfinite(incl_cos))
        return fail(M2M_ERR_ARG, "weight_scale must be finite and > 0; inclination finite");

    // tables on the host, checked against the fixed capacity
    PassArgs a;
    memset(&a, 0, sizeof a);
    std::vector<float> edges, gh;
    int nobs = 0;
    for (int s = 0; s < nsets; ++s) {
        const m2m_obs_desc &o = obs[s];
        SetDev &d = a.sets[s];
        d.geom = o.geom; d.quant = o.quant; d.nx = o.nx; d.ny = o.geom == M2M_GEOM_GRID ? o.ny : 1;
        if (o.geom < 1 || o.geom > 3 || o.quant < 1 || o.quant > 3 || o.nx < 1 || d.ny < 1 || !o.edges_x ||
            (o.geom == M2M_GEOM_GRID && !o.edges_y) || o.psf_q)
            return fail(M2M_ERR_ARG, "observable set %d: bad geometry/quantity/sizes/edges", s);
        d.nmom = o.quant == M2M_Q_GH ? 5 : 1;
        d.gx_top = (float)(d.nx - 1);
        d.gy_top = (float)(d.ny - 1);
        const long long cells = (long long)d.nx * d.ny;
        d.ncell = (int)cells;
        d.obs_off = nobs;
        if (nobs + cells * d.nmom > M2M_STATIC_MAX_OBS)
            return fail(M2M_ERR_ARG, "more than %d observables (the static scratch capacity)", M2M_STATIC_MAX_OBS);
        nobs += (int)(cells * d.nmom);
        for (int ax = 0; ax < (o.geom == M2M_GEOM_GRID ? 2 : 1); ++ax) {
            const double *e = ax == 0 ? o.edges_x : o.edges_y;
            const int nb = ax == 0 ? d.nx : d.ny;
            if ((long long)edges.size() + nb + 1 > M2M_STATIC_MAX_EDGES)
                return fail(M2M_ERR_ARG, "more than %d edges in total (the static scratch capacity)",
                            M2M_STATIC_MAX_EDGES);
            for (int k = 0; k <= nb; ++k)
                if (!(e[k] == e[k]) || (k > 0 && !(e[k] > e[k - 1])))
                    return fail(M2M_ERR_ARG, "observable set %d: edges must be strictly increasing", s);
            const int off = (int)edges.size();
            for (int k = 0; k <= nb; ++k) edges.push_back(ceil_float(e[k]));
            if (ax == 0) { d.ex_off = off; guess_params(e, nb, &d.gx_mode, &d.gx_a, &d.gx_b); }
            else { d.ey_off = off; guess_params(e, nb, &d.gy_mode, &d.gy_a, &d.gy_b); }
        }
        if (o.quant == M2M_Q_GH) {
            if (!o.gh_V || !o.gh_S || !(o.sigma_kernel >= 0))
                return fail(M2M_ERR_ARG, "observable set %d: GH needs gh_V, gh_S, sigma_kernel>=0", s);
            if ((long long)gh.size() / 5 + cells > M2M_STATIC_MAX_GH_CELLS)
                return fail(M2M_ERR_ARG, "more than %d Gauss-Hermite cells (the static scratch capacity)",
                            M2M_STATIC_MAX_GH_CELLS);
            d.gh_off = (int)gh.size();
            d.ghc_off = d.gh_off / 5;
            for (long long c = 0; c < cells; ++c) {
                const double S = o.gh_S[c];
                if (!(S > 0) || !isfinite(o.gh_V[c])) return fail(M2M_ERR_ARG, "observable set %d: gh_S must be > 0", s);
                const double sk = o.sigma_kernel / S, d1 = 1.0 + sk * sk;
                gh.push_back((float)o.gh_V[c]);
                gh.push_back((float)(1.0 / S));
                gh.push_back((float)(1.0 / d1));
                gh.push_back((float)(sk * sk / d1));
                gh.push_back((float)(2.0 * sqrt(M_PI) / sqrt(2.0 * M_PI * d1)));
            }
        }
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(M2M_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(M2M_ERR_ARG, "device %d beyond %d", dev, MAX_DEVICES);
    int rc = setup_device(dev);
    if (rc) return rc;
    unsigned char *base = g_scratch_ptr[dev];

    // tables into the scratch (pageable sources: the copies have consumed
    // them when the calls return), totals and error word cleared
    e = cudaMemcpyAsync(base + OFF_EDGES, edges.data(), 4 * edges.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !gh.empty())
        e = cudaMemcpyAsync(base + OFF_GH, gh.data(), 4 * gh.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + OFF_TOT, 0, 8ull * nobs, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + OFF_ERR, 0, 4, st);
    if (e != cudaSuccess) return fail(M2M_ERR_CUDA, "scratch upload: %s", cudaGetErrorString(e));

    // the scatter pass of m2m_observe: FP32C, 1024 threads, no cell cache;
    // the fixed-point scale of a context: 2^-25 of the average weight
    // weight_scale / n (both rounded up to powers of two)
    // (sums within 1e-12 above a power of two taken as that power, as for
    // contexts)
    const int wexp = (int)ceil(log2(weight_scale * (1.0 - 1e-12)));
    int nbits = 0;
    while ((1ll << nbits) < n) ++nbits;
    a.x = (void *)x; a.y = (void *)y; a.z = (void *)z; a.vx = (void *)vx; a.vy = (void *)vy; a.vz = (void *)vz;
    a.w = (double *)w; a.what = (double *)w;
    a.n = n; a.flags = F_SCAT; a.nsets = nsets; a.nobs = nobs; a.npot = 0;
    a.sin_i = incl_sin; a.cos_i = incl_cos;
    a.f_sin_i = (float)incl_sin; a.f_cos_i = (float)incl_cos;
    a.edge_tab = base + OFF_EDGES; a.edge_len = (int)edges.size();
    a.gh_tab = base + OFF_GH; a.gh_len = (int)gh.size();
    a.fx_shift = FX_AVG_BITS + nbits - wexp;
    a.y_acc = (unsigned long long *)(base + OFF_TOT);
    a.fx_atomic = 1;
    a.err = (int *)(base + OFF_ERR);
    a.prior_kind = M2M_PRIOR_FLAT; a.nE = 1; a.nL = 1;
    const int layout = layout_of(a.sets, nsets);
    void *fn = pass_kernel_f32(1024, layout);
    const size_t sm = pass_smem_bytes(true, layout, F_SCAT, nobs, a.edge_len, a.gh_len, 0, 1, 1, 0);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 1024, sm);
    if (e != cudaSuccess || occ < 1) return fail(M2M_ERR_CUDA, "scatter does not fit: %s", cudaGetErrorString(e));
    long long grid = (long long)g_nsm[dev] * occ;
    const long long need = (n + 1023) / 1024;
    if (grid > need) grid = need;
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(1024), args, sm, st);
    if (e != cudaSuccess) return fail(M2M_ERR_CUDA, "scatter launch: %s", cudaGetErrorString(e));
    k_static_finish<<<(nobs + 127) / 128, 128, 0, st>>>(a.y_acc, a.err, y_out, nobs, ldexp(1.0, -a.fx_shift));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(M2M_ERR_CUDA, "finish launch: %s", cudaGetErrorString(e));
    return M2M_OK;
}

}  // extern "C"
