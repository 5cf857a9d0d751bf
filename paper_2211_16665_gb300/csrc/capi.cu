// Host side of the C ABI declared in include/csem.h: context set-up (grid
// widths, CFL step, CPML recursion tables, transform weights), point
// operators, and the run loop that replays CUDA-graph chunks of time steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/csem.h"
#include "csem_internal.cuh"
#include "csem_td.cuh"
#include "csem_ho.cuh"
#include "csem_es.cuh"

using csem::C2;
using csem::Tap;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? CSEM_ERR_OOM : CSEM_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

constexpr double kMu0 = 4e-7 * M_PI;
constexpr double kCpmlR = 1e-6;
constexpr double kDecaySpan = 35.0;
constexpr int kChunk = 64;        // time steps per captured graph
constexpr int kMaxSide = 4;       // event slots for overlapped flushes (at most two are in flight)
constexpr int kEsDepth = 4;       // early end: chunks in flight before the host reads a convergence flag

struct Axis {
    int n = 0;
    std::vector<double> x, h, ht;   // nodes, primal widths (n), dual widths (n+1)
    std::vector<double> bh, ah, bn, an;
    std::vector<double> wh, wn;     // fourth order: [n][4] at half nodes, [n+1][4] at nodes
};

// Derivative at x0 of the Lagrange interpolant through the four points x[0..3]:
// w_i = L_i'(x0) = sum_{m != i} 1/(x_i - x_m) prod_{l != i, m} (x0 - x_l)/(x_i - x_l).
void lagrange_d1(double x0, const double *x, double *w) {
    for (int i = 0; i < 4; ++i) {
        double sum = 0.0;
        for (int m = 0; m < 4; ++m) {
            if (m == i) continue;
            double prod = 1.0 / (x[i] - x[m]);
            for (int l = 0; l < 4; ++l)
                if (l != i && l != m) prod *= (x0 - x[l]) / (x[i] - x[l]);
            sum += prod;
        }
        w[i] = sum;
    }
}

// Fourth-order staggered weights of one axis (Sec. 2, high-order differences on the
// non-uniform grid): the half node p from the nodes p-1 .. p+2 and the node q from
// the half nodes q-2 .. q+1, each exact for cubics; two-point rows where four points
// do not fit (half nodes 0 and n-1, nodes 1 and n-1).  Returns the largest absolute
// row sum touching a cell (the bound of the difference's symbol, for the CFL step).
double ho_axis(Axis &A) {
    const int n = A.n;
    A.wh.assign(4 * (size_t)n, 0.0);
    A.wn.assign(4 * (size_t)(n + 1), 0.0);
    std::vector<double> xh(n);
    for (int i = 0; i < n; ++i) xh[i] = 0.5 * (A.x[i] + A.x[i + 1]);
    for (int p = 0; p < n; ++p) {
        if (p >= 1 && p <= n - 2) lagrange_d1(xh[p], &A.x[p - 1], &A.wh[4 * p]);
        else { A.wh[4 * p + 1] = -1.0 / A.h[p]; A.wh[4 * p + 2] = 1.0 / A.h[p]; }
    }
    for (int q = 1; q < n; ++q) {
        if (q >= 2 && q <= n - 2) lagrange_d1(A.x[q], &xh[q - 2], &A.wn[4 * q]);
        else { A.wn[4 * q + 1] = -1.0 / A.ht[q]; A.wn[4 * q + 2] = 1.0 / A.ht[q]; }
    }
    auto rs = [](const double *w) { return std::fabs(w[0]) + std::fabs(w[1]) + std::fabs(w[2]) + std::fabs(w[3]); };
    double smax = 0.0;
    for (int i = 0; i < n; ++i)
        smax = std::max(smax, std::max(rs(&A.wh[4 * i]), std::max(rs(&A.wn[4 * i]), rs(&A.wn[4 * (i + 1)]))));
    return smax;
}

// CPML recursion coefficients psi <- b psi + a du (Komatitsch & Martin 2007 with
// kappa = 1): d = d0 (xi/L)^2, d0 = -3 v ln(R) / (2 L), alpha = pi f0 (1 - xi/L),
// b = exp(-(d + alpha) dt), a = d (b - 1) / (d + alpha); zero outside the layer.
void cpml_axis(Axis &A, int npml, double dt, double v, double f0) {
    const int n = A.n;
    A.bh.assign(n, 0.0); A.ah.assign(n, 0.0); A.bn.assign(n + 1, 0.0); A.an.assign(n + 1, 0.0);
    if (npml == 0) return;
    const double lo = A.x[npml], hi = A.x[n - npml];
    const double Llo = lo - A.x[0], Lhi = A.x[n] - hi;
    auto eval = [&](double p, double &b, double &a) {
        double xi = 0.0, L = 1.0;
        if (p < lo) { xi = lo - p; L = Llo; }
        else if (p > hi) { xi = p - hi; L = Lhi; }
        if (!(xi > 0.0)) { b = 0.0; a = 0.0; return; }
        const double d0 = -3.0 * v * std::log(kCpmlR) / (2.0 * L);
        const double d = d0 * (xi / L) * (xi / L);
        const double al = M_PI * f0 * (1.0 - xi / L);
        b = std::exp(-(d + al) * dt);
        a = d * (b - 1.0) / (d + al);
    };
    for (int i = 0; i < n; ++i) eval(0.5 * (A.x[i] + A.x[i + 1]), A.bh[i], A.ah[i]);
    for (int i = 0; i <= n; ++i) eval(A.x[i], A.bn[i], A.an[i]);
}

}  // namespace

namespace csem {
int set_last_error(int code, const std::string &msg) { return fail(code, msg); }
}  // namespace csem

struct csem_ctx {
    int device = 0;
    int nx, ny, nz, npml, NX, NY, NZ, pitch;
    long long plane, vol;
    Axis ax[3];
    double f0, w0, rho_max, dt, safety;
    int nt, precision, kahan, nf, max_src, max_rec;
    int vti = 0;                         // 1: models [2][cells] = (rho_h, rho_v), gradients (h, v)
    int order = 2;                       // spatial order of the differences: 2 (Yee) or 4
    void *d_ho = nullptr;                // fourth order: weight tables (real) wxh|wxn|wyh|wyn|wzh|wzn
    std::vector<double> freqs, a;        // a_k = sqrt(w_k w0)
    std::vector<std::complex<double>> kf, alpha_fwd;
    std::vector<double> wavelet;         // J'(t_{n+1/2})
    int KZ_h = 4, KZ_e = 4;             // z planes per thread (autotuned)
    int MB_h = 4, MB_e = 4;             // min resident blocks per SM of the compiled variant (autotuned)
    int fused_kz = 0;                   // > 0: fused H+E step with this z blocking (autotuned)
    int FZ_by = 0, FZ_mb = 4, FZ_kz = 16; // FZ_by > 0: fused one-pass FP32 step, rows per block (autotuned)
    int FZ_ws = 0;                        // 1: the warp-specialised fused step with those shape fields
    int WAVE_lag = 0, WAVE_kz = 4, WAVE_mb = 8; // WAVE_lag > 0: wave-ordered FP32 step (autotuned)
    int fault_tx = 0;                   // test hook: extra bytes the bulk-copy kernels' first barrier arm expects
    int VEC_h = 0, VEC_e = 0;           // 1: four-cells-per-thread FP32 kernels (autotuned)
    int TMA_h = 0, TMA_e = 0;           // > 0: bulk-copy-staged FP32 kernels, rows per block (autotuned)
    int LEAN_h = 0, LEAN_e = 0;         // > 0: lean FP32 kernels, cells per thread (autotuned; needs d_psiL)
    long long psi_stride = 0, sx = 0, sy = 0, sz = 0;
    size_t rsize = 4;
    // device memory
    void *d_tab = nullptr;               // per-axis stepping tables (real)
    double *d_h = nullptr;               // primal widths (double) hx|hy|hz
    void *d_tabL = nullptr;              // padded FP32 stepping tables (lean kernels)
    float *d_psiL = nullptr, *d_cEm = nullptr;   // lean kernels: CPML memory in volume arrays, masked dt/eps
    float *d_q = nullptr;                // fused one-pass step: V sigma per cell [1 or 2][vol] (sigma_h, sigma_v)
    float *d_tabG = nullptr;             // fused one-pass step: per-axis widths h [n] and sums s [n+1], padded
    unsigned *d_wave = nullptr;          // wave-ordered step: ticket, finished-block and per-z-block counters
    void *d_cE = nullptr, *d_H = nullptr, *d_H2 = nullptr, *d_ering = nullptr, *d_psi = nullptr, *d_comp = nullptr, *d_edge = nullptr;
    int M = 16, nslot = 17;
    int flush_mode = 0;                  // bit 0: bulk-copy flush (FP32 only), else register flush;
                                         // bit 1: flush on the side stream, overlapping the next block

    void *d_wR = nullptr;                // [nt][nf] complex real
    double2 *d_w64 = nullptr;            // [nt][nf]
    double2 *d_alpha = nullptr;          // [0..nf): forward, [nf..2nf): adjoint, [2nf..3nf): k_f
    double2 *d_racc = nullptr;
    double *d_coef = nullptr, *d_T = nullptr, *d_ones = nullptr;
    Tap *d_rtaps = nullptr, *d_itaps = nullptr;
    int2 *d_colmap = nullptr;            // [max_src][plane] injection taps per lattice column
    unsigned char *d_tflag = nullptr;    // [max(max_src, max_rec)][ny][nseg] columns with taps, per 32 along x
    int nseg = 1;
    float *d_inc = nullptr;              // lean kernels: [kChunk][max_src][ntl] tap increments of a chunk
    int *d_tapk = nullptr;               // [max(max_src, max_rec) * 8] plane * 4 + component of each tap
    int last_ntl = 8;                    // taps per list of the last run (8 forward, 8 * receivers adjoint)
    bool last_shared = false;            // the uploaded taps are an adjoint run's (one list, receiver emitters)
    long long *d_cpos = nullptr;         // scatter positions / values for the column map
    int2 *d_cval = nullptr;
    int *d_step = nullptr, *d_bad = nullptr;
    double *d_trace = nullptr;
    int last_nrec = 0;
    long long bytes = 0;
    cudaStream_t cap = nullptr, side = nullptr;
    cudaEvent_t ev_fork[kMaxSide] = {}, ev_done[kMaxSide] = {};
    // early end of forward data runs (tol > 0): previous and kept receiver transforms,
    // device state {ended, steps}, host copies of the ended flag per chunk slot
    double es_tol = 0.0;
    double2 *d_rprev = nullptr, *d_rfin = nullptr;
    int *d_es = nullptr, *h_es = nullptr;
    cudaEvent_t es_ev[kEsDepth] = {};
    bool last_es = false;                // the last forward or adjoint run used an early end
    // early end of runs that keep volumes (tol > 0): previous accumulators, per-frequency stats
    double es_vol_tol = 0.0;
    double es_vol_floor = 1e-4;          // entries below this fraction of their frequency's largest: absolute bound
    void *d_vprev = nullptr;             // [max_src][3][nf][vol] complex (real)
    unsigned *d_vstats = nullptr;        // [3 nf]: max |acc|, moved flag, previous check's max
    struct GraphSlot { int key[8]; cudaGraphExec_t exec; };
    std::vector<GraphSlot> graphs;
};

namespace {

template <typename T>
int dalloc(csem_ctx *c, T **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CSEM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    c->bytes += (long long)bytes;
    return CSEM_OK;
}

#define TRY(x)                  \
    do {                        \
        int r_ = (x);           \
        if (r_ != CSEM_OK) return r_; \
    } while (0)

template <typename R>
void axis_tab(const csem_ctx *c, int a, csem::AxisTab<R> &t) {
    const R *base = (const R *)c->d_tab;
    long long off = 0;
    for (int b = 0; b < a; ++b) off += 6LL * (c->ax[b].n + 1);
    const int n = c->ax[a].n;
    t.ih_h = base + off;
    t.ih_n = base + off + (n + 1);
    t.b_h = base + off + 2 * (n + 1);
    t.a_h = base + off + 3 * (n + 1);
    t.b_n = base + off + 4 * (n + 1);
    t.a_n = base + off + 5 * (n + 1);
}

// Lean-kernel tables: per axis ih_h, ih_n, b_h, a_h, b_n, a_n, each padded to
// lean_len(n) floats (16-byte groups, zero past the axis); b_n, a_n are zero on
// the outer nodes 0 and n, which carry no CPML update.
int lean_len(int n) { return (n + 1 + 3 + 3) / 4 * 4; }
// The fused one-pass step's launch shape as one code (0: not selected): kz * 100 + rows * 10 + blocks;
// csem_autotune and csem_set_launch report and take it as 10000 + that code.
// The wave-ordered step (kern_lean.cu) takes 40000 + lag * 100 + planes * 10 + blocks.
int fz_code(const csem_ctx *c) {
    if (c->WAVE_lag) return 40000 + c->WAVE_lag * 100 + c->WAVE_kz * 10 + c->WAVE_mb;
    return c->FZ_by ? c->FZ_ws * 20000 + c->FZ_kz * 100 + c->FZ_by * 10 + c->FZ_mb : 0;
}
// Per-axis widths of the fused one-pass step: h (primal, half nodes) and s = h[i-1] + h[i] at the
// nodes (the outer nodes take their one width), each padded to lean_len(n) floats.
int upload_geo_tables(csem_ctx *c) {
    std::vector<float> tab;
    for (int a = 0; a < 3; ++a) {
        const Axis &A = c->ax[a];
        const int n = A.n, L = lean_len(n);
        std::vector<float> v(2 * (size_t)L, 0.f);
        for (int i = 0; i < n; ++i) v[i] = (float)A.h[i];
        for (int i = 0; i <= n; ++i) v[L + i] = (float)((i > 0 ? A.h[i - 1] : 0.0) + (i < n ? A.h[i] : 0.0));
        tab.insert(tab.end(), v.begin(), v.end());
    }
    TRY(dalloc(c, &c->d_tabG, tab.size() * sizeof(float)));
    CK(cudaMemcpy(c->d_tabG, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice));
    return CSEM_OK;
}
void lean_tab(const csem_ctx *c, int a, csem::AxisTab<float> &t) {
    const float *base = (const float *)c->d_tabL;
    long long off = 0;
    for (int b = 0; b < a; ++b) off += 6LL * lean_len(c->ax[b].n);
    const int L = lean_len(c->ax[a].n);
    t.ih_h = base + off; t.ih_n = base + off + L; t.b_h = base + off + 2 * L;
    t.a_h = base + off + 3 * L; t.b_n = base + off + 4 * L; t.a_n = base + off + 5 * L;
}
int upload_lean_tables(csem_ctx *c) {
    std::vector<float> tab;
    for (int a = 0; a < 3; ++a) {
        const Axis &A = c->ax[a];
        const int n = A.n, L = lean_len(n);
        std::vector<float> v(6 * (size_t)L, 0.f);
        for (int i = 0; i < n; ++i) {
            v[i] = (float)(1.0 / A.h[i]);
            v[2 * L + i] = (float)A.bh[i];
            v[3 * L + i] = (float)A.ah[i];
        }
        for (int i = 0; i <= n; ++i) v[L + i] = (float)(1.0 / A.ht[i]);
        for (int i = 1; i < n; ++i) { v[4 * L + i] = (float)A.bn[i]; v[5 * L + i] = (float)A.an[i]; }
        tab.insert(tab.end(), v.begin(), v.end());
    }
    tab.insert(tab.end(), 4, 0.f);   // zeros read by lanes off the x slab
    TRY(dalloc(c, &c->d_tabL, tab.size() * sizeof(float)));
    CK(cudaMemcpy(c->d_tabL, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice));
    return CSEM_OK;
}

template <typename R>
int upload_tables(csem_ctx *c) {
    std::vector<R> tab;
    for (int a = 0; a < 3; ++a) {
        const Axis &A = c->ax[a];
        const int n = A.n;
        std::vector<R> ih_h(n + 1, R(0)), ih_n(n + 1, R(0)), bh(n + 1, R(0)), ah(n + 1, R(0)), bn(n + 1), an(n + 1);
        for (int i = 0; i < n; ++i) { ih_h[i] = (R)(1.0 / A.h[i]); bh[i] = (R)A.bh[i]; ah[i] = (R)A.ah[i]; }
        for (int i = 0; i <= n; ++i) { ih_n[i] = (R)(1.0 / A.ht[i]); bn[i] = (R)A.bn[i]; an[i] = (R)A.an[i]; }
        for (auto *v : {&ih_h, &ih_n, &bh, &ah, &bn, &an}) tab.insert(tab.end(), v->begin(), v->end());
    }
    TRY(dalloc(c, (R **)&c->d_tab, tab.size() * sizeof(R)));
    CK(cudaMemcpy(c->d_tab, tab.data(), tab.size() * sizeof(R), cudaMemcpyHostToDevice));
    // transform weights exp((-1 + i) a_k n dt), n = 0..nt-1  (Eq. 6)
    std::vector<typename C2<R>::T> wR((size_t)c->nt * c->nf);
    std::vector<double2> w64((size_t)c->nt * c->nf);
    for (int n = 0; n < c->nt; ++n)
        for (int f = 0; f < c->nf; ++f) {
            const double t = n * c->dt;
            const double e = std::exp(-c->a[f] * t);
            const double re = e * std::cos(c->a[f] * t), im = e * std::sin(c->a[f] * t);
            w64[(size_t)n * c->nf + f] = make_double2(re, im);
            wR[(size_t)n * c->nf + f].x = (R)re;
            wR[(size_t)n * c->nf + f].y = (R)im;
        }
    TRY(dalloc(c, (typename C2<R>::T **)&c->d_wR, wR.size() * sizeof(wR[0])));
    CK(cudaMemcpy(c->d_wR, wR.data(), wR.size() * sizeof(wR[0]), cudaMemcpyHostToDevice));
    TRY(dalloc(c, &c->d_w64, w64.size() * sizeof(double2)));
    CK(cudaMemcpy(c->d_w64, w64.data(), w64.size() * sizeof(double2), cudaMemcpyHostToDevice));
    return CSEM_OK;
}

// forward normalisation alpha_k = k_k / What_k with What_k the damped transform
// of the wavelet at the injection times (n + 1/2) dt (Eq. 3 and Eq. 6)
int update_wavelet(csem_ctx *c) {
    c->alpha_fwd.assign(c->nf, 0.0);
    for (int f = 0; f < c->nf; ++f) {
        std::complex<double> W(0.0, 0.0);
        for (int n = 0; n < c->nt; ++n) {
            if (c->wavelet[n] == 0.0) continue;
            const double t = (n + 0.5) * c->dt;
            W += c->wavelet[n] * std::exp(std::complex<double>(-c->a[f] * t, c->a[f] * t));
        }
        if (std::abs(W) == 0.0) return fail(CSEM_ERR_INVALID_ARG, "wavelet has a zero transform at a frequency");
        c->alpha_fwd[f] = c->kf[f] / W;
    }
    std::vector<double2> al(3 * c->nf);
    for (int f = 0; f < c->nf; ++f) {
        al[f] = make_double2(c->alpha_fwd[f].real(), c->alpha_fwd[f].imag());
        al[c->nf + f] = make_double2(c->dt, 0.0);
        al[2 * c->nf + f] = make_double2(c->kf[f].real(), c->kf[f].imag());
    }
    CK(cudaMemcpy(c->d_alpha, al.data(), al.size() * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_T, c->wavelet.data(), c->nt * sizeof(double), cudaMemcpyHostToDevice));
    return CSEM_OK;
}

// Trilinear taps of a point on component comp's lattice.  inject: divide by the edge's dual volume.
int point_taps(const csem_ctx *c, double px, double py, double pz, int comp, bool inject, int emit, Tap *out) {
    if (comp < 0 || comp > 2) return fail(CSEM_ERR_INVALID_ARG, "point component must be 0, 1 or 2");
    const double p[3] = {px, py, pz};
    int lo[3];
    double wt[3][2];
    for (int a = 0; a < 3; ++a) {
        const Axis &A = c->ax[a];
        const bool half = (a == comp);
        const int len = half ? A.n : A.n + 1;
        auto g = [&](int m) { return half ? 0.5 * (A.x[m] + A.x[m + 1]) : A.x[m]; };
        if (!std::isfinite(p[a])) return fail(CSEM_ERR_OUT_OF_DOMAIN, "non-finite point coordinate");
        int m = 0;
        {   // largest m with g(m) <= p, clamped to [0, len-2]
            int l = 0, r = len - 1;
            while (r - l > 1) { int mid = (l + r) / 2; if (g(mid) <= p[a]) l = mid; else r = mid; }
            m = l;
        }
        const double t = (p[a] - g(m)) / (g(m + 1) - g(m));
        if (t < -1e-9 || t > 1.0 + 1e-9) return fail(CSEM_ERR_OUT_OF_DOMAIN, "point outside the grid");
        lo[a] = m;
        wt[a][0] = 1.0 - t;
        wt[a][1] = t;
    }
    int q = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = lo[0] + di, j = lo[1] + dj, k = lo[2] + dk;
                double w = wt[0][di] * wt[1][dj] * wt[2][dk];
                // an edge on the outer boundary is never updated: only zero weights may land there
                bool upd = true;
                if (comp == 0) upd = (j >= 1 && j < c->ny && k >= 1 && k < c->nz);
                if (comp == 1) upd = (i >= 1 && i < c->nx && k >= 1 && k < c->nz);
                if (comp == 2) upd = (i >= 1 && i < c->nx && j >= 1 && j < c->ny);
                if (!upd) {
                    if (std::fabs(w) > 1e-12) return fail(CSEM_ERR_OUT_OF_DOMAIN, "point touches the outer boundary");
                    w = 0.0;
                }
                if (inject && w != 0.0) {
                    const Axis &X = c->ax[0], &Y = c->ax[1], &Z = c->ax[2];
                    double dV = 0.0;
                    if (comp == 0) dV = X.h[i] * Y.ht[j] * Z.ht[k];
                    if (comp == 1) dV = X.ht[i] * Y.h[j] * Z.ht[k];
                    if (comp == 2) dV = X.ht[i] * Y.ht[j] * Z.h[k];
                    w /= dV;
                }
                Tap &tp = out[q++];
                tp.idx = ((long long)k * c->NY + j) * c->pitch + i;
                tp.w = w;
                tp.comp = comp;
                tp.emit = emit;
                tp.pad0 = tp.pad1 = 0;
            }
    return CSEM_OK;
}

int check_points(const csem_points *p, int max_n, const char *what, bool allow_empty) {
    if (!p) return fail(CSEM_ERR_INVALID_ARG, std::string(what) + " is NULL");
    if (p->n < (allow_empty ? 0 : 1) || p->n > max_n)
        return fail(CSEM_ERR_INVALID_ARG, std::string(what) + " count out of range");
    if (p->n > 0 && (!p->x || !p->y || !p->z || !p->comp))
        return fail(CSEM_ERR_INVALID_ARG, std::string(what) + " has NULL arrays");
    return CSEM_OK;
}

template <typename R>
csem::StepParams<R> step_params(csem_ctx *c, bool dft, void *acc) {
    csem::StepParams<R> p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz; p.NX = c->NX; p.NY = c->NY; p.NZ = c->NZ;
    p.pitch = c->pitch; p.npml = c->npml; p.plane = c->plane; p.vol = c->vol;
    axis_tab<R>(c, 0, p.ax); axis_tab<R>(c, 1, p.ay); axis_tab<R>(c, 2, p.az);
    p.H = (R *)c->d_H;
    p.H2 = (R *)c->d_H2;
    p.fused_kz = c->fused_kz;
    p.ering = (R *)c->d_ering;
    p.ering_stride = (long long)c->nslot * 3 * c->vol;
    p.nslot = c->nslot;
    p.psi = (R *)c->d_psi;
    p.psi_stride = c->psi_stride; p.sx = c->sx; p.sy = c->sy; p.sz = c->sz;
    p.cE = (const R *)c->d_cE;
    p.cH = (R)(c->dt / kMu0);
    p.step = c->d_step;
    p.KZ_h = c->KZ_h;
    p.KZ_e = c->KZ_e;
    p.MB_h = c->MB_h;
    p.MB_e = c->MB_e;
    p.VEC_h = c->VEC_h;
    p.VEC_e = c->VEC_e;
    p.TMA_h = c->TMA_h;
    p.TMA_e = c->TMA_e;
    p.LEAN_h = c->LEAN_h;
    p.LEAN_e = c->LEAN_e;
    p.lx = p.ly = p.lz = csem::AxisTab<R>{};
    p.lzero = nullptr;
    p.FZ_by = 0; p.FZ_mb = 4; p.FZ_kz = 16; p.FZ_ws = 0;
    p.WAVE_lag = 0; p.WAVE_kz = 4; p.WAVE_mb = 8;
    p.wave = nullptr;
    p.qh = p.qv = nullptr;
    p.gx = p.gy = p.gz = csem::GeoTab{nullptr, nullptr};
    p.k2w0dt = 0.f;
    p.inc = nullptr;
    p.tapk = nullptr;
    p.psiL = nullptr;
    p.cEm = nullptr;
    if constexpr (sizeof(R) == 4) {
        if (c->d_tabL) {
            lean_tab(c, 0, p.lx); lean_tab(c, 1, p.ly); lean_tab(c, 2, p.lz);
            long long off = 0;
            for (int a = 0; a < 3; ++a) off += 6LL * lean_len(c->ax[a].n);
            p.lzero = (const float *)c->d_tabL + off;
        }
        p.psiL = c->d_psiL;
        p.cEm = c->d_cEm;
        p.wave = c->d_wave;
        if (c->d_wave && c->d_psiL) { p.WAVE_lag = c->WAVE_lag; p.WAVE_kz = c->WAVE_kz; p.WAVE_mb = c->WAVE_mb; }
        p.inc = c->d_inc;
        p.tapk = c->d_tapk;
        if (c->d_q && c->d_tabG) {
            p.FZ_by = c->FZ_by; p.FZ_mb = c->FZ_mb; p.FZ_kz = c->FZ_kz; p.FZ_ws = c->FZ_ws;
            p.qh = c->d_q;
            p.qv = c->vti ? c->d_q + c->vol : c->d_q;
            const csem::GeoTab *g[3] = {&p.gx, &p.gy, &p.gz};
            long long off = 0;
            for (int a = 0; a < 3; ++a) {
                const int L = lean_len(c->ax[a].n);
                const_cast<csem::GeoTab *>(g[a])->h = c->d_tabG + off;
                const_cast<csem::GeoTab *>(g[a])->s = c->d_tabG + off + L;
                off += 2LL * L;
            }
            p.k2w0dt = (float)(2.0 * c->w0 * c->dt);
        }
    }
    p.err = c->d_bad;
    p.fault_tx = c->fault_tx;
    p.colmap = nullptr;
    p.colmap_stride = 0;
    p.tflag = nullptr;
    p.tflag_stride = 0;
    p.nseg = c->nseg;
    p.inc_ntl = 0;
    p.itaps = nullptr;
    p.itap_stride = 0;
    p.n_emit = p.J = 0;
    p.coef = p.T = nullptr;
    p.nf = c->nf;
    p.w = (const typename C2<R>::T *)c->d_wR;
    p.acc = dft ? (typename C2<R>::T *)acc : nullptr;
    p.comp = (dft && c->kahan) ? (typename C2<R>::T *)c->d_comp : nullptr;
    return p;
}

// Zeroes the state of S sources (H, the E ring, the CPML memory) and the step counter.
template <typename R>
int reset_state(csem_ctx *c, int S, cudaStream_t st) {
    CK(cudaMemsetAsync(c->d_H, 0, (size_t)S * 3 * c->vol * sizeof(R), st));
    CK(cudaMemsetAsync(c->d_H2, 0, (size_t)S * 3 * c->vol * sizeof(R), st));
    CK(cudaMemsetAsync(c->d_ering, 0, (size_t)S * c->nslot * 3 * c->vol * sizeof(R), st));
    CK(cudaMemsetAsync(c->d_psi, 0, (size_t)S * c->psi_stride * sizeof(R), st));
    if (c->d_psiL) CK(cudaMemsetAsync(c->d_psiL, 0, (size_t)S * 12 * c->vol * sizeof(float), st));
    CK(cudaMemsetAsync(c->d_step, 0, sizeof(int), st));
    return CSEM_OK;
}

// One transform flush of cnt snapshots: the bulk-copy kernel when selected and
// applicable (FP32, volumes, a whole block), else the register kernel.
template <typename R>
cudaError_t flush(csem_ctx *c, const csem::StepParams<R> &p, const csem::PointParams<R> &q, int S, int n0_off,
                  int cnt, bool vol, bool kahan, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if ((c->flush_mode & 1) && vol && (cnt == 16 || cnt == 32 || cnt == 64 || cnt == 128))
            return csem::launch_dft_bulk(p, q, S, n0_off, cnt, kahan, c->d_bad, st);
    }
    return csem::launch_dft<R>(p, q, S, n0_off, cnt, vol, kahan, st);
}

template <typename R>
csem::HoTab<R> ho_tab(const csem_ctx *c) {
    const R *t = (const R *)c->d_ho;
    csem::HoTab<R> w;
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    w.wxh = t; w.wxn = w.wxh + 4 * nx;
    w.wyh = w.wxn + 4 * (nx + 1); w.wyn = w.wyh + 4 * ny;
    w.wzh = w.wyn + 4 * (ny + 1); w.wzn = w.wzh + 4 * nz;
    return w;
}

// One step (or its H / E half, which: bit 0 H, bit 2 E) with the kernels of the context's order.
template <typename R>
cudaError_t launch_any(const csem_ctx *c, const csem::StepParams<R> &p, const csem::PointParams<R> &q, int S,
                       int jstep, cudaStream_t st, int which = 5) {
    if (c->order == 4) return csem::launch_ho<R>(p, ho_tab<R>(c), S, jstep, st, which);
    return csem::launch_step<R>(p, q, S, jstep, st, which);
}

// Tap increments of the next nsteps steps for the lean E kernel (FP32 runs with injection).
template <typename R>
cudaError_t tap_prep(csem_ctx *c, const csem::StepParams<R> &p, int S, int nsteps, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if (p.inc && p.colmap && (p.LEAN_e || p.FZ_by || p.WAVE_lag)) return csem::launch_tap_inc(p, S, nsteps, c->nt, st);
    }
    return cudaSuccess;
}

// Steps 0 .. n-1 (relative to the device step counter) with a transform flush
// after every M steps.  Without overlap each flush follows its block on st.
// With overlap (flush_mode bit 1) the flush of block b runs on the side stream
// while block b+1 steps, and st waits for it before the first step of block b+2,
// the first step that rewrites one of its ring slots (nslot >= 2M + 1).  lead:
// first flush the block that ended just before step 0 (skipped on the device
// when that block would start before step 0); trail: flush the last block here
// too, else it is left for the next call's lead.  Flushes run one after another
// on one stream in block order either way, so the results do not depend on the
// overlap.
template <typename R>
cudaError_t emit_steps(csem_ctx *c, int S, bool vol, bool kahan, const csem::StepParams<R> &p,
                       const csem::PointParams<R> &q, int n, bool lead, bool trail, cudaStream_t st) {
    const int M = c->M;
    const bool overlap = (c->flush_mode & 2) != 0;
    // side flushes in flight: event slot k % kMaxSide, due before step join_at[k];
    // at most two are in flight, so a slot is joined before it is recorded again
    int nev = 0, njoined = 0;
    int join_at[kMaxSide];
    auto join = [&](int j) -> cudaError_t {   // every side flush due before step j, oldest first
        while (njoined < nev && join_at[njoined % kMaxSide] <= j) {
            cudaError_t e = cudaStreamWaitEvent(st, c->ev_done[njoined % kMaxSide], 0);
            if (e != cudaSuccess) return e;
            ++njoined;
        }
        return cudaSuccess;
    };
    auto side_flush = [&](int n0_off) -> cudaError_t {
        if (nev - njoined >= kMaxSide) return cudaErrorInvalidValue;
        const int k = nev % kMaxSide;
        cudaError_t e = cudaEventRecord(c->ev_fork[k], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork[k], 0);
        if (e == cudaSuccess) e = flush<R>(c, p, q, S, n0_off, M, vol, kahan, c->side);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_done[k], c->side);
        join_at[k] = n0_off + 2 * M;
        ++nev;
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (lead) e = overlap ? side_flush(-M) : flush<R>(c, p, q, S, -M, M, vol, kahan, st);
    for (int j = 0; j < n && e == cudaSuccess; ++j) {
        if (overlap) e = join(j);
        if (e == cudaSuccess) e = launch_any<R>(c, p, q, S, j, st);
        if (e != cudaSuccess || (j + 1) % M != 0 || (j + 1 == n && !trail)) continue;
        e = overlap ? side_flush(j + 1 - M) : flush<R>(c, p, q, S, j + 1 - M, M, vol, kahan, st);
    }
    if (e == cudaSuccess && overlap) e = join(1 << 30);
    return e;
}

// Captures one chunk of launches (emit on the capture stream) into a graph and
// returns the executable kept for key (updated in place when only parameters
// changed) and the number of kernels one replay launches.
template <typename Emit>
int chunk_graph(csem_ctx *c, const int key[8], Emit &&emit, cudaGraphExec_t *out, long long *per_chunk) {
    cudaGraph_t g = nullptr;
    const long long before = csem::g_launches.load();   // captured kernels are counted per replay
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = emit(c->cap);
    cudaError_t ee = cudaStreamEndCapture(c->cap, &g);
    if (le != cudaSuccess) return fail(CSEM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(le));
    CK(ee);
    cudaGraphExec_t exec = nullptr;
    for (auto &slot : c->graphs)
        if (std::equal(key, key + 8, slot.key)) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(slot.exec, g, &info) == cudaSuccess) exec = slot.exec;
            else {
                cudaGetLastError();
                CK(cudaDeviceSynchronize());
                cudaGraphExecDestroy(slot.exec);
                CK(cudaGraphInstantiate(&slot.exec, g, 0));
                exec = slot.exec;
            }
            break;
        }
    if (!exec) {
        csem_ctx::GraphSlot slot;
        std::copy(key, key + 8, slot.key);
        CK(cudaGraphInstantiate(&slot.exec, g, 0));
        c->graphs.push_back(slot);
        exec = slot.exec;
    }
    cudaGraphDestroy(g);
    *per_chunk = csem::g_launches.load() - before;
    csem::g_launches -= *per_chunk;
    *out = exec;
    return CSEM_OK;
}

// nt steps of H, E and injection; after every M steps the finished snapshots are
// transformed (and the receivers sampled).  Full chunks of kChunk steps replay
// one captured graph; the remainder and the final partial block are launched
// directly.  With overlapped flushes a chunk's last block is flushed at the start
// of the next chunk (or of the remainder).
template <typename R>
int run_steps(csem_ctx *c, int S, bool vol, const csem::StepParams<R> &p, const csem::PointParams<R> &q,
              cudaStream_t st) {
    const bool kahan = vol && c->kahan;
    const int M = c->M;
    const bool overlap = (c->flush_mode & 2) != 0;
    const int full = c->nt / kChunk, rem = c->nt % kChunk;
    // M = 2 kChunk (never overlapped): chunks alternate between a graph without a flush and one
    // that ends with the flush of both chunks' snapshots
    const bool two = M > kChunk;
    int pending = 0;                // steps before the device counter not yet transformed
    if (full > 0) {
        int key[8] = {S, vol ? 1 : 0, kahan ? 1 : 0, (q.n_itaps > 0 ? 1 : 0) + 2 * fz_code(c), q.n_rec > 0 ? 1 : 0,
                      (int)sizeof(R), ((c->KZ_h * 16 + c->KZ_e) * 16 + c->MB_h) * 16 + c->MB_e,
                      ((((M * 4 + c->flush_mode) * 32 + c->fused_kz) * 4 + c->VEC_h * 2 + c->VEC_e) * 25 +
                       c->TMA_h * 5 + c->TMA_e) * 16 + c->LEAN_h * 4 + c->LEAN_e};
        cudaGraphExec_t exec = nullptr, exec2 = nullptr;
        long long per_chunk = 0, per_chunk2 = 0;
        TRY(chunk_graph(c, key, [&](cudaStream_t cs) {
            cudaError_t le = tap_prep<R>(c, p, S, kChunk, cs);
            if (le == cudaSuccess) le = emit_steps<R>(c, S, vol, kahan, p, q, kChunk, overlap, !overlap, cs);
            if (le == cudaSuccess) le = csem::launch_advance(c->d_step, kChunk, cs);
            return le;
        }, &exec, &per_chunk));
        if (two) {
            key[1] += 2;            // the second graph of the pair
            TRY(chunk_graph(c, key, [&](cudaStream_t cs) {
                cudaError_t le = tap_prep<R>(c, p, S, kChunk, cs);
                if (le == cudaSuccess) le = emit_steps<R>(c, S, vol, kahan, p, q, kChunk, false, true, cs);
                if (le == cudaSuccess) le = flush<R>(c, p, q, S, kChunk - M, M, vol, kahan, cs);
                if (le == cudaSuccess) le = csem::launch_advance(c->d_step, kChunk, cs);
                return le;
            }, &exec2, &per_chunk2));
        }
        for (int ch = 0; ch < full; ++ch) {
            const bool second = two && (ch % 2 == 1);
            CK(cudaGraphLaunch(second ? exec2 : exec, st));
            csem::g_launches += second ? per_chunk2 : per_chunk;
        }
        if (overlap) CK(flush<R>(c, p, q, S, -M, M, vol, kahan, st));
        if (two && full % 2 == 1) pending = kChunk;
    }
    auto emit = [&](int j, cudaStream_t s2) -> cudaError_t {
        cudaError_t e = launch_any<R>(c, p, q, S, j, s2);
        if (e == cudaSuccess && (pending + j + 1) % M == 0) e = flush<R>(c, p, q, S, j + 1 - M, M, vol, kahan, s2);
        return e;
    };
    if (rem > 0) CK(tap_prep<R>(c, p, S, rem, st));
    for (int j = 0; j < rem; ++j) CK(emit(j, st));
    const int tail = (pending + rem) % M;   // the steps after the last whole block
    if (tail) CK(flush<R>(c, p, q, S, rem - tail, tail, vol, kahan, st));
    return CSEM_OK;
}

csem::GeoD geo(const csem_ctx *c) {
    csem::GeoD g;
    g.nx = c->nx; g.ny = c->ny; g.nz = c->nz; g.NX = c->NX; g.NY = c->NY; g.NZ = c->NZ;
    g.pitch = c->pitch; g.plane = c->plane; g.vol = c->vol;
    g.hx = c->d_h; g.hy = c->d_h + c->nx; g.hz = c->d_h + c->nx + c->ny;
    return g;
}

// dt/eps on every E edge from the model (and, for the lean kernels, its copy with
// the PEC edges zeroed).
template <typename R>
int coef_init(csem_ctx *c, const void *rho, cudaStream_t st) {
    const long long cells = (long long)c->nx * c->ny * c->nz;
    const R *rho_h = (const R *)rho, *rho_z = rho_h + (c->vti ? cells : 0);
    CK(csem::launch_coef_init<R>(geo(c), rho_h, rho_z, (R *)c->d_cE, 2.0 * c->w0 * c->dt, c->d_bad, st));
    if constexpr (sizeof(R) == 4) {
        if (c->d_cEm) CK(csem::launch_mask_coef(step_params<float>(c, false, nullptr), (const float *)c->d_cE, c->d_cEm, st));
        if (c->d_q) CK(csem::launch_qcell(geo(c), (const float *)rho_h, (const float *)rho_z, c->d_q,
                                          c->vti ? c->d_q + c->vol : nullptr, st));
    }
    return CSEM_OK;
}

// Device arrays that describe one injection (the context's own, or a second set).
struct InjDst {
    Tap *itaps;
    int2 *colmap;
    unsigned char *tflag;
    int *tapk;
};

// Sorts each source's injection taps by lattice column (then index) and sets the
// device column map: colmap[s*stride + col] = (first tap, count), zero elsewhere.
// dst: where to put the taps, column map, tile flags and tap planes (NULL: the context's).
int upload_injection(csem_ctx *c, std::vector<Tap> &taps, int n_lists, int per_list, bool shared, cudaStream_t st,
                     const InjDst *dst = nullptr) {
    const InjDst own{c->d_itaps, c->d_colmap, c->d_tflag, c->d_tapk};
    const InjDst &d = dst ? *dst : own;
    const long long plane = c->plane;
    std::vector<long long> pos;
    std::vector<int2> val;
    for (int s = 0; s < n_lists; ++s) {
        auto b = taps.begin() + (size_t)s * per_list;
        std::stable_sort(b, b + per_list, [&](const Tap &x, const Tap &y) {
            const long long cx = x.idx % plane, cy = y.idx % plane;
            return cx != cy ? cx < cy : x.idx < y.idx;
        });
        for (int u = 0; u < per_list; ++u) {
            const long long col = b[u].idx % plane;
            if (u == 0 || (b[u - 1].idx % plane) != col) {
                pos.push_back((shared ? 0 : (long long)s * plane) + col);
                val.push_back(make_int2(u, 0));
            }
            val.back().y += 1;
        }
    }
    CK(cudaMemcpyAsync(d.itaps, taps.data(), taps.size() * sizeof(Tap), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d.colmap, 0, (size_t)(shared ? 1 : n_lists) * plane * sizeof(int2), st));
    CK(cudaMemcpyAsync(c->d_cpos, pos.data(), pos.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_cval, val.data(), val.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(csem::launch_scatter_int2(d.colmap, c->d_cpos, c->d_cval, (int)pos.size(), st));
    {   // tile flags: rows and 32-column segments of the cell range that hold a tap
        const int nl = shared ? 1 : n_lists;
        std::vector<unsigned char> fl((size_t)nl * c->ny * c->nseg, 0);
        for (int s = 0; s < n_lists; ++s)
            for (int u = 0; u < per_list; ++u) {
                const long long col = taps[(size_t)s * per_list + u].idx % plane;
                const int j = (int)(col / c->pitch), i = (int)(col % c->pitch);
                if (j < c->ny && i < c->nx) fl[((size_t)(shared ? 0 : s) * c->ny + j) * c->nseg + i / 32] = 1;
            }
        CK(cudaMemcpyAsync(d.tflag, fl.data(), fl.size(), cudaMemcpyHostToDevice, st));
    }
    if (d.tapk) {   // plane and component of each tap, for the lean E kernel
        std::vector<int> tk(taps.size());
        for (size_t u = 0; u < taps.size(); ++u) tk[u] = (int)(taps[u].idx / plane) * 4 + taps[u].comp;
        CK(cudaMemcpyAsync(d.tapk, tk.data(), tk.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    if (!dst) {
        c->last_ntl = per_list;
        c->last_shared = shared;
    }
    return CSEM_OK;
}

// Forward data run with the early end (Sec. 2): whole chunks replay the captured
// graph (block flushes in order, no overlap), each followed by the convergence
// check; the host keeps at most kEsDepth chunks in flight and stops issuing once a
// check it has read says the run has ended (chunks already issued then run, but
// the kept spectra are those of the ending chunk).  Without an end the remainder
// runs as in run_steps and the last check keeps the full transform.
template <typename R>
int run_steps_es(csem_ctx *c, int S, int NR, const csem::StepParams<R> &p, const csem::PointParams<R> &q,
                 cudaStream_t st) {
    const int saved = c->flush_mode, savedM = c->M;
    c->flush_mode &= 1;
    c->M = std::min(c->M, kChunk);       // a check after every chunk: whole blocks within a chunk
    struct Restore { csem_ctx *c; int m, M; ~Restore() { c->flush_mode = m; c->M = M; } } restore{c, saved, savedM};
    const int M = c->M, nt = c->nt, n = S * NR * c->nf;
    const int full = nt / kChunk, rem = nt % kChunk;
    CK(cudaMemsetAsync(c->d_es, 0, 2 * sizeof(int), st));
    bool ended = false;
    if (full > 0) {
        const int key[8] = {S, 4, fz_code(c), q.n_itaps > 0 ? 1 : 0, 1, (int)sizeof(R),
                            ((c->KZ_h * 16 + c->KZ_e) * 16 + c->MB_h) * 16 + c->MB_e,
                            ((((M * 4 + c->flush_mode) * 32 + c->fused_kz) * 4 + c->VEC_h * 2 + c->VEC_e) * 25 +
                             c->TMA_h * 5 + c->TMA_e) * 16 + c->LEAN_h * 4 + c->LEAN_e};
        cudaGraphExec_t exec = nullptr;
        long long per_chunk = 0;
        TRY(chunk_graph(c, key, [&](cudaStream_t cs) {
            cudaError_t le = tap_prep<R>(c, p, S, kChunk, cs);
            if (le == cudaSuccess) le = emit_steps<R>(c, S, false, false, p, q, kChunk, false, true, cs);
            if (le == cudaSuccess) le = csem::launch_advance(c->d_step, kChunk, cs);
            return le;
        }, &exec, &per_chunk));
        for (int ch = 0; ch < full; ++ch) {
            const int slot = ch % kEsDepth;
            if (ch >= kEsDepth) {
                CK(cudaEventSynchronize(c->es_ev[slot]));
                if (c->h_es[slot]) { ended = true; break; }
            }
            CK(cudaGraphLaunch(exec, st));
            csem::g_launches += per_chunk;
            const bool last = (ch == full - 1 && rem == 0);
            CK(csem::launch_es_check(c->d_racc, c->d_rprev, c->d_rfin, n, c->es_tol, ch, last ? 1 : 0,
                                     (ch + 1) * kChunk, c->d_es, st));
            CK(cudaMemcpyAsync(&c->h_es[slot], c->d_es, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaEventRecord(c->es_ev[slot], st));
        }
    }
    if (!ended && rem > 0) {
        CK(tap_prep<R>(c, p, S, rem, st));
        for (int j = 0; j < rem; ++j) {
            CK(launch_any<R>(c, p, q, S, j, st));
            if ((j + 1) % M == 0) CK(flush<R>(c, p, q, S, j + 1 - M, M, false, false, st));
        }
        const int tail = rem % M;
        if (tail) CK(flush<R>(c, p, q, S, rem - tail, tail, false, false, st));
        CK(csem::launch_es_check(c->d_racc, c->d_rprev, c->d_rfin, n, c->es_tol, full, 1, nt, c->d_es, st));
    }
    return CSEM_OK;
}

// A run that keeps volumes, with the early end (Sec. 2): after every chunk of
// kChunk steps (graph replay, block flushes in order) one pass over the transform
// accumulators gives, per frequency, the largest magnitude and the largest change
// since the previous check; the run ends after the first chunk c >= 1 whose changes
// are all within tol of the magnitudes.  The host reads each chunk's verdict before
// issuing the next chunk, so no step after the end touches the volumes or the
// receivers.  Without an end the remainder runs as in run_steps.
template <typename R>
int run_steps_vol_es(csem_ctx *c, int S, const csem::StepParams<R> &p, const csem::PointParams<R> &q,
                     cudaStream_t st) {
    typedef typename C2<R>::T R2;
    const int saved = c->flush_mode, savedM = c->M;
    c->flush_mode &= 1;
    c->M = std::min(c->M, kChunk);       // a check after every chunk: whole blocks within a chunk
    struct Restore { csem_ctx *c; int m, M; ~Restore() { c->flush_mode = m; c->M = M; } } restore{c, saved, savedM};
    const bool kahan = c->kahan != 0;
    const int M = c->M, nt = c->nt, nf = c->nf;
    const int full = nt / kChunk, rem = nt % kChunk;
    CK(cudaMemsetAsync(c->d_es, 0, 2 * sizeof(int), st));
    CK(cudaMemsetAsync(c->d_vstats, 0, 3 * nf * sizeof(unsigned), st));
    // the transform weights fall by q = exp((-1 + i) a_k kChunk dt) per chunk (Eq. 6): a field
    // that stays as it was over the last chunk adds |q| / |1 - q| times that chunk's change
    csem::EsTail tail{};
    for (int f = 0; f < nf; ++f) {
        const std::complex<double> q = std::exp(std::complex<double>(-1.0, 1.0) * (c->a[f] * kChunk * c->dt));
        tail.f[f] = (float)(std::abs(q) / std::abs(1.0 - q));
    }
    bool ended = false;
    if (full > 0) {
        const int key[8] = {S, 5, (kahan ? 1 : 0) + 2 * fz_code(c), q.n_itaps, q.n_rec > 0 ? 1 : 0, (int)sizeof(R),
                            ((c->KZ_h * 16 + c->KZ_e) * 16 + c->MB_h) * 16 + c->MB_e,
                            ((((M * 4 + c->flush_mode) * 32 + c->fused_kz) * 4 + c->VEC_h * 2 + c->VEC_e) * 25 +
                             c->TMA_h * 5 + c->TMA_e) * 16 + c->LEAN_h * 4 + c->LEAN_e};
        cudaGraphExec_t exec = nullptr;
        long long per_chunk = 0;
        TRY(chunk_graph(c, key, [&](cudaStream_t cs) {
            cudaError_t le = tap_prep<R>(c, p, S, kChunk, cs);
            if (le == cudaSuccess) le = emit_steps<R>(c, S, true, kahan, p, q, kChunk, false, true, cs);
            if (le == cudaSuccess) le = csem::launch_advance(c->d_step, kChunk, cs);
            return le;
        }, &exec, &per_chunk));
        for (int ch = 0; ch < full; ++ch) {
            CK(cudaGraphLaunch(exec, st));
            csem::g_launches += per_chunk;
            const bool last = (ch == full - 1 && rem == 0);
            CK(cudaMemsetAsync(c->d_vstats, 0, 2 * nf * sizeof(unsigned), st));
            CK(csem::launch_es_vol_stats<R>((const R2 *)p.acc, (R2 *)c->d_vprev, c->vol, S, nf, c->es_vol_tol,
                                            c->es_vol_floor, tail, c->d_vstats, st));
            CK(csem::launch_es_vol_decide(c->d_vstats, nf, ch, last ? 1 : 0, (ch + 1) * kChunk, c->d_es, st));
            CK(cudaMemcpyAsync(&c->h_es[0], c->d_es, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaEventRecord(c->es_ev[0], st));
            CK(cudaEventSynchronize(c->es_ev[0]));
            if (c->h_es[0]) { ended = true; break; }
        }
    }
    if (!ended && rem > 0) {
        CK(tap_prep<R>(c, p, S, rem, st));
        for (int j = 0; j < rem; ++j) {
            CK(launch_any<R>(c, p, q, S, j, st));
            if ((j + 1) % M == 0) CK(flush<R>(c, p, q, S, j + 1 - M, M, true, kahan, st));
        }
        const int tail = rem % M;
        if (tail) CK(flush<R>(c, p, q, S, rem - tail, tail, true, kahan, st));
        CK(csem::launch_es_vol_decide(c->d_vstats, nf, full, 1, nt, c->d_es, st));
    }
    return CSEM_OK;
}

template <typename R>
int fwd_impl(csem_ctx *c, const void *rho, const csem_points *src, const csem_points *rec, double *d_syn,
             void *Evol, cudaStream_t st) {
    const int S = src->n, NR = rec->n;
    std::vector<Tap> itaps((size_t)S * 8), rtaps((size_t)std::max(NR, 1) * 8);
    for (int s = 0; s < S; ++s)
        TRY(point_taps(c, src->x[s], src->y[s], src->z[s], src->comp[s], true, 0, &itaps[(size_t)s * 8]));
    for (int r = 0; r < NR; ++r)
        TRY(point_taps(c, rec->x[r], rec->y[r], rec->z[r], rec->comp[r], false, r, &rtaps[(size_t)r * 8]));
    TRY(upload_injection(c, itaps, S, 8, false, st));
    if (NR > 0) CK(cudaMemcpyAsync(c->d_rtaps, rtaps.data(), (size_t)NR * 8 * sizeof(Tap), cudaMemcpyHostToDevice, st));
    TRY(coef_init<R>(c, rho, st));
    TRY(reset_state<R>(c, S, st));
    const bool dft = (Evol != nullptr);
    const size_t vbytes = (size_t)S * 3 * c->nf * c->vol * sizeof(typename C2<R>::T);
    if (dft) CK(cudaMemsetAsync(Evol, 0, vbytes, st));
    if (dft && c->kahan) CK(cudaMemsetAsync(c->d_comp, 0, vbytes, st));
    if (NR > 0) CK(cudaMemsetAsync(c->d_racc, 0, (size_t)S * NR * c->nf * sizeof(double2), st));
    if (c->d_trace && NR > 0) CK(cudaMemsetAsync(c->d_trace, 0, (size_t)S * NR * c->nt * sizeof(double), st));

    csem::StepParams<R> p = step_params<R>(c, dft, Evol);
    p.colmap = c->d_colmap; p.colmap_stride = c->plane;
    p.tflag = c->d_tflag; p.tflag_stride = (long long)c->ny * c->nseg;
    p.inc_ntl = 8;
    p.itaps = c->d_itaps; p.itap_stride = 8;
    p.n_emit = 1; p.J = 1; p.coef = c->d_ones; p.T = c->d_T;   // unit moment for every source
    csem::PointParams<R> q;
    q.cE = (const R *)c->d_cE; q.step = c->d_step;
    q.nt = c->nt; q.nf = c->nf;
    q.n_rec = NR; q.rtaps = c->d_rtaps; q.racc = c->d_racc; q.w64 = c->d_w64; q.trace = c->d_trace;
    q.n_itaps = 8; q.itaps = c->d_itaps; q.itap_stride = 8;
    q.n_emit = 1; q.J = 1; q.coef = c->d_ones; q.T = c->d_T;
    const bool es = c->es_tol > 0.0 && NR > 0 && !dft;
    const bool es_vol = c->es_vol_tol > 0.0 && dft;
    if (es) TRY(run_steps_es<R>(c, S, NR, p, q, st));
    else if (es_vol) TRY(run_steps_vol_es<R>(c, S, p, q, st));
    else TRY(run_steps<R>(c, S, dft, p, q, st));
    c->last_es = es || es_vol;
    c->last_nrec = NR;
    if (NR > 0)
        CK(csem::launch_finalize_receivers(es ? c->d_rfin : c->d_racc, d_syn, S, NR, c->nf, c->d_alpha, st));
    if (dft)
        CK(csem::launch_finalize_volume<R>((typename C2<R>::T *)Evol,
                                           c->kahan ? (const typename C2<R>::T *)c->d_comp : nullptr, c->vol, S,
                                           c->nf, c->d_alpha, st));
    return CSEM_OK;
}

template <typename R>
int adj_impl(csem_ctx *c, const void *rho, const csem_points *rec, int S, const double *resid, const double *basis,
             void *Vvol, cudaStream_t st) {
    const int NR = rec->n;
    std::vector<Tap> itaps((size_t)NR * 8);
    for (int r = 0; r < NR; ++r)
        TRY(point_taps(c, rec->x[r], rec->y[r], rec->z[r], rec->comp[r], true, r, &itaps[(size_t)r * 8]));
    TRY(upload_injection(c, itaps, 1, NR * 8, true, st));
    CK(csem::launch_adjoint_coef(resid, c->d_coef, S, NR, c->nf, c->d_alpha + 2 * c->nf, 1.0 / c->dt, st));
    TRY(coef_init<R>(c, rho, st));
    TRY(reset_state<R>(c, S, st));
    const size_t vbytes = (size_t)S * 3 * c->nf * c->vol * sizeof(typename C2<R>::T);
    CK(cudaMemsetAsync(Vvol, 0, vbytes, st));
    if (c->kahan) CK(cudaMemsetAsync(c->d_comp, 0, vbytes, st));
    csem::StepParams<R> p = step_params<R>(c, true, Vvol);
    p.colmap = c->d_colmap; p.colmap_stride = 0;
    p.tflag = c->d_tflag; p.tflag_stride = 0;
    p.inc_ntl = NR * 8;
    p.itaps = c->d_itaps; p.itap_stride = 0;
    p.n_emit = NR; p.J = 2 * c->nf; p.coef = c->d_coef; p.T = basis;
    csem::PointParams<R> q;
    q.cE = (const R *)c->d_cE; q.step = c->d_step;
    q.nt = c->nt; q.nf = c->nf;
    q.n_rec = 0; q.rtaps = nullptr; q.racc = nullptr; q.w64 = c->d_w64; q.trace = nullptr;
    q.n_itaps = NR * 8; q.itaps = c->d_itaps; q.itap_stride = 0;
    q.n_emit = NR; q.J = 2 * c->nf; q.coef = c->d_coef; q.T = basis;
    const bool es_vol = c->es_vol_tol > 0.0;
    if (es_vol) TRY(run_steps_vol_es<R>(c, S, p, q, st));
    else TRY(run_steps<R>(c, S, true, p, q, st));
    c->last_es = es_vol;
    CK(csem::launch_finalize_volume<R>((typename C2<R>::T *)Vvol,
                                       c->kahan ? (const typename C2<R>::T *)c->d_comp : nullptr, c->vol, S, c->nf,
                                       c->d_alpha + c->nf, st));
    return CSEM_OK;
}

// ---------------------------------------------------------------------------
// Time-domain adjoint gradient (appendix).  The forward run is cut into
// segments of C steps.  A first pass steps segments 0 .. K-2 and keeps the
// state at each segment start 1 .. K-2 (checkpoints).  The sweep then takes the
// segments last to first: it steps the forward segment again from its start
// (the last one continues from the first pass, the first one from zero), so that
// E^{n_a} .. E^{n_b} sit in a ring of C + 1 snapshots, and advances the adjoint
// run (reversed time) over the matching m range in sub-blocks of up to B steps,
// each followed by the correlation of its B snapshots with the forward ring.
// Forward steps: (K - 1) C + nt; adjoint steps: nt.
// ---------------------------------------------------------------------------
struct TdPlan {
    int C = 0, K = 0, B = kChunk, nck = 0;
    bool lean = false, fused = false;
    size_t o_seg = 0, o_aH = 0, o_aH2 = 0, o_aring = 0, o_apsi = 0, o_apsiL = 0, o_T = 0, o_coef = 0, o_acc = 0;
    size_t o_itaps = 0, o_colmap = 0, o_tflag = 0, o_tapk = 0, o_ck = 0;
    size_t ck_H = 0, ck_E = 0, ck_psi = 0, ck_psiL = 0, ck_bytes = 0, total = 0;
    long long recompute = 0;             // forward steps beyond nt
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

TdPlan td_layout(const csem_ctx *c, int S, int NR, int C) {
    TdPlan P;
    P.C = C;
    P.K = (c->nt + C - 1) / C;
    P.nck = std::max(P.K - 2, 0);
    P.recompute = (long long)(P.K - 1) * C;
    P.lean = c->d_psiL && (c->LEAN_h || c->LEAN_e || c->WAVE_lag) && !c->FZ_by;
    P.fused = c->fused_kz > 0 || c->FZ_by > 0;
    const size_t R = c->rsize, v3 = 3 * (size_t)c->vol, Ss = (size_t)S;
    const size_t psi = Ss * (size_t)c->psi_stride * R, psiL = P.lean ? Ss * 12 * (size_t)c->vol * sizeof(float) : 0;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += al256(bytes); return at; };
    P.o_seg = take(Ss * (size_t)(C + 1) * v3 * R);
    P.o_aH = take(Ss * v3 * R);
    P.o_aH2 = take(P.fused ? Ss * v3 * R : 0);
    P.o_aring = take(Ss * (size_t)(P.B + 1) * v3 * R);
    P.o_apsi = take(psi);
    P.o_apsiL = take(psiL);
    P.o_T = take((size_t)c->nt * 2 * c->nf * sizeof(double));
    P.o_coef = take(Ss * NR * 2 * c->nf * sizeof(double));
    P.o_acc = take(v3 * sizeof(double));
    P.o_itaps = take((size_t)NR * 8 * sizeof(Tap));
    P.o_colmap = take((size_t)c->plane * sizeof(int2));
    P.o_tflag = take((size_t)c->ny * c->nseg);
    P.o_tapk = take(c->d_tapk ? (size_t)NR * 8 * sizeof(int) : 0);
    P.o_ck = o;
    size_t q = 0;
    auto ck = [&](size_t bytes) { const size_t at = q; q += al256(bytes); return at; };
    P.ck_H = ck(Ss * v3 * R);
    P.ck_E = ck(Ss * v3 * R);
    P.ck_psi = ck(psi);
    P.ck_psiL = ck(psiL);
    P.ck_bytes = q;
    P.total = o + (size_t)P.nck * P.ck_bytes;
    return P;
}

// segment > 0: that length (even); else the candidate with the least forward
// recomputation whose workspace fits budget (budget <= 0: the least workspace).
int td_plan(const csem_ctx *c, int S, int NR, int segment, long long budget, TdPlan *out) {
    if (segment > 0) {
        if (segment % 2) return fail(CSEM_ERR_INVALID_ARG, "segment length must be even");
        *out = td_layout(c, S, NR, segment);
        return CSEM_OK;
    }
    std::vector<TdPlan> cand;
    cand.push_back(td_layout(c, S, NR, (c->nt + 1) / 2 * 2));              // whole run, no recomputation
    for (int K = 2; K <= (c->nt + kChunk - 1) / kChunk; ++K) {
        const int C = ((c->nt + K - 1) / K + kChunk - 1) / kChunk * kChunk;
        if ((c->nt + C - 1) / C == K) cand.push_back(td_layout(c, S, NR, C));
    }
    const TdPlan *best = nullptr;
    for (const auto &P : cand) {
        if (budget > 0) {
            if ((long long)P.total > budget) continue;
            if (!best || P.recompute < best->recompute || (P.recompute == best->recompute && P.total < best->total))
                best = &P;
        } else if (!best || P.total < best->total) {
            best = &P;
        }
    }
    if (!best) return fail(CSEM_ERR_OOM, "no checkpoint plan fits the workspace budget");
    *out = *best;
    return CSEM_OK;
}

// Steps n0 .. n0+L-1 of one run without transforms: whole chunks of kChunk steps
// replay a graph captured per role (2: forward, 3: adjoint) on first use, the
// rest is launched directly.
struct RoleGraph {
    cudaGraphExec_t exec = nullptr;
    long long per_chunk = 0;
};

template <typename R>
int run_range(csem_ctx *c, int S, int role, RoleGraph &g, const csem::StepParams<R> &p,
              const csem::PointParams<R> &q, int n0, int L, cudaStream_t st) {
    CK(csem::launch_set_step(c->d_step, n0, st));
    const int full = L / kChunk, rem = L % kChunk;
    if (full > 0 && !g.exec) {
        const int key[8] = {S, role, fz_code(c), q.n_itaps, q.n_emit, (int)sizeof(R),
                            ((c->KZ_h * 16 + c->KZ_e) * 16 + c->MB_h) * 16 + c->MB_e,
                            (((c->fused_kz * 4 + c->VEC_h * 2 + c->VEC_e) * 25 + c->TMA_h * 5 + c->TMA_e) * 16 +
                             c->LEAN_h * 4 + c->LEAN_e)};
        TRY(chunk_graph(c, key, [&](cudaStream_t cs) {
            cudaError_t e = tap_prep<R>(c, p, S, kChunk, cs);
            for (int j = 0; j < kChunk && e == cudaSuccess; ++j) e = launch_any<R>(c, p, q, S, j, cs);
            if (e == cudaSuccess) e = csem::launch_advance(c->d_step, kChunk, cs);
            return e;
        }, &g.exec, &g.per_chunk));
    }
    for (int ch = 0; ch < full; ++ch) {
        CK(cudaGraphLaunch(g.exec, st));
        csem::g_launches += g.per_chunk;
    }
    if (rem > 0) {
        CK(tap_prep<R>(c, p, S, rem, st));
        for (int j = 0; j < rem; ++j) CK(launch_any<R>(c, p, q, S, j, st));
    }
    return CSEM_OK;
}

template <typename R>
int td_impl(csem_ctx *c, const void *rho, const csem_points *src, const csem_points *rec, const double *resid,
            int segment, int wrt, void *grad, void *work, long long work_bytes, cudaStream_t st) {
    const int S = src->n, NR = rec->n, nt = c->nt;
    TdPlan P;
    TRY(td_plan(c, S, NR, segment, 0, &P));
    if (work_bytes < (long long)P.total)
        return fail(CSEM_ERR_INVALID_ARG, "workspace of " + std::to_string(work_bytes) + " bytes, the plan needs " +
                                              std::to_string((long long)P.total));
    if ((uintptr_t)work % 256) return fail(CSEM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    char *w = (char *)work;
    const size_t v3 = 3 * (size_t)c->vol, R_ = sizeof(R);
    const int C = P.C, B = P.B;

    // injection: the sources into the forward run (the context's arrays), the
    // receivers as emitters of the adjoint run (the workspace's)
    std::vector<Tap> itaps((size_t)S * 8), rtaps((size_t)NR * 8);
    for (int s = 0; s < S; ++s)
        TRY(point_taps(c, src->x[s], src->y[s], src->z[s], src->comp[s], true, 0, &itaps[(size_t)s * 8]));
    for (int r = 0; r < NR; ++r)
        TRY(point_taps(c, rec->x[r], rec->y[r], rec->z[r], rec->comp[r], true, r, &rtaps[(size_t)r * 8]));
    TRY(upload_injection(c, itaps, S, 8, false, st));
    const InjDst adst{(Tap *)(w + P.o_itaps), (int2 *)(w + P.o_colmap), (unsigned char *)(w + P.o_tflag),
                      c->d_tapk ? (int *)(w + P.o_tapk) : nullptr};
    TRY(upload_injection(c, rtaps, 1, NR * 8, true, st, &adst));
    TRY(coef_init<R>(c, rho, st));
    double *T = (double *)(w + P.o_T), *coef = (double *)(w + P.o_coef), *acc = (double *)(w + P.o_acc);
    CK(csem::launch_td_series(c->d_w64, T, nt, c->nf, st));
    CK(csem::launch_td_coef(resid, c->d_alpha, coef, S, NR, c->nf, st));

    // zero state: forward (context arrays; its E lives in the segment ring), adjoint, accumulator
    R *seg = (R *)(w + P.o_seg), *aring = (R *)(w + P.o_aring);
    const long long seg_stride = (long long)(C + 1) * v3, a_stride = (long long)(B + 1) * v3;
    const size_t psi_b = (size_t)S * c->psi_stride * R_, psiL_b = P.lean ? (size_t)S * 12 * c->vol * sizeof(float) : 0;
    auto zero_forward = [&]() -> int {
        CK(cudaMemsetAsync(c->d_H, 0, (size_t)S * v3 * R_, st));
        if (psi_b) CK(cudaMemsetAsync(c->d_psi, 0, psi_b, st));
        if (psiL_b) CK(cudaMemsetAsync(c->d_psiL, 0, psiL_b, st));
        CK(cudaMemset2DAsync(seg, seg_stride * R_, 0, v3 * R_, S, st));      // E^0 in slot 0
        return CSEM_OK;
    };
    TRY(zero_forward());
    // the kernels never write the row padding and the PEC boundary edges, so every slot starts at zero
    CK(cudaMemsetAsync(seg, 0, (size_t)S * seg_stride * R_, st));
    CK(cudaMemsetAsync(w + P.o_aH, 0, (size_t)S * v3 * R_, st));
    if (P.fused) CK(cudaMemsetAsync(w + P.o_aH2, 0, (size_t)S * v3 * R_, st));
    CK(cudaMemsetAsync(aring, 0, (size_t)S * a_stride * R_, st));
    if (psi_b) CK(cudaMemsetAsync(w + P.o_apsi, 0, psi_b, st));
    if (psiL_b) CK(cudaMemsetAsync(w + P.o_apsiL, 0, psiL_b, st));
    CK(cudaMemsetAsync(acc, 0, v3 * sizeof(double), st));

    csem::StepParams<R> pf = step_params<R>(c, false, nullptr);
    pf.ering = seg; pf.ering_stride = seg_stride; pf.nslot = C + 1;
    pf.colmap = c->d_colmap; pf.colmap_stride = c->plane;
    pf.tflag = c->d_tflag; pf.tflag_stride = (long long)c->ny * c->nseg;
    pf.inc_ntl = 8;
    pf.itaps = c->d_itaps; pf.itap_stride = 8;
    pf.n_emit = 1; pf.J = 1; pf.coef = c->d_ones; pf.T = c->d_T;
    csem::PointParams<R> qf;
    qf.cE = (const R *)c->d_cE; qf.step = c->d_step;
    qf.nt = nt; qf.nf = c->nf;
    qf.n_rec = 0; qf.rtaps = nullptr; qf.racc = nullptr; qf.w64 = c->d_w64; qf.trace = nullptr;
    qf.n_itaps = 8; qf.itaps = c->d_itaps; qf.itap_stride = 8;
    qf.n_emit = 1; qf.J = 1; qf.coef = c->d_ones; qf.T = c->d_T;

    csem::StepParams<R> pa = step_params<R>(c, false, nullptr);
    pa.H = (R *)(w + P.o_aH); pa.H2 = P.fused ? (R *)(w + P.o_aH2) : pa.H;
    pa.ering = aring; pa.ering_stride = a_stride; pa.nslot = B + 1;
    pa.psi = (R *)(w + P.o_apsi);
    if constexpr (sizeof(R) == 4) pa.psiL = P.lean ? (float *)(w + P.o_apsiL) : nullptr;
    pa.colmap = adst.colmap; pa.colmap_stride = 0;
    pa.tflag = adst.tflag; pa.tflag_stride = 0;
    pa.inc_ntl = NR * 8;
    if constexpr (sizeof(R) == 4) pa.tapk = adst.tapk;
    pa.itaps = adst.itaps; pa.itap_stride = 0;
    pa.n_emit = NR; pa.J = 2 * c->nf; pa.coef = coef; pa.T = T;
    csem::PointParams<R> qa = qf;
    qa.n_itaps = NR * 8; qa.itaps = adst.itaps; qa.itap_stride = 0;
    qa.n_emit = NR; qa.J = 2 * c->nf; qa.coef = coef; qa.T = T;

    // checkpoint j (1 .. K-2) holds the forward state at n = j C
    auto ck_at = [&](int j) { return w + P.o_ck + (size_t)(j - 1) * P.ck_bytes; };
    auto save = [&](int j) -> int {
        char *d = ck_at(j);
        const int sl = (j * C) % (C + 1);
        CK(cudaMemcpyAsync(d + P.ck_H, c->d_H, (size_t)S * v3 * R_, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpy2DAsync(d + P.ck_E, v3 * R_, seg + (size_t)sl * v3, seg_stride * R_, v3 * R_, S,
                             cudaMemcpyDeviceToDevice, st));
        if (psi_b) CK(cudaMemcpyAsync(d + P.ck_psi, c->d_psi, psi_b, cudaMemcpyDeviceToDevice, st));
        if (psiL_b) CK(cudaMemcpyAsync(d + P.ck_psiL, c->d_psiL, psiL_b, cudaMemcpyDeviceToDevice, st));
        return CSEM_OK;
    };
    auto restore = [&](int j) -> int {
        const char *d = ck_at(j);
        const int sl = (j * C) % (C + 1);
        CK(cudaMemcpyAsync(c->d_H, d + P.ck_H, (size_t)S * v3 * R_, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpy2DAsync(seg + (size_t)sl * v3, seg_stride * R_, d + P.ck_E, v3 * R_, v3 * R_, S,
                             cudaMemcpyDeviceToDevice, st));
        if (psi_b) CK(cudaMemcpyAsync(c->d_psi, d + P.ck_psi, psi_b, cudaMemcpyDeviceToDevice, st));
        if (psiL_b) CK(cudaMemcpyAsync(c->d_psiL, d + P.ck_psiL, psiL_b, cudaMemcpyDeviceToDevice, st));
        return CSEM_OK;
    };

    // first pass: segments 0 .. K-2, keeping the starts of segments 1 .. K-2
    RoleGraph gf, ga;
    for (int k = 0; k + 1 < P.K; ++k) {
        TRY(run_range<R>(c, S, 2, gf, pf, qf, k * C, C, st));
        if (k + 1 <= P.K - 2) TRY(save(k + 1));
    }
    // sweep: last segment first; the adjoint advances through m = 0 .. nt-1 in order
    for (int k = P.K - 1; k >= 0; --k) {
        const int na = k * C, L = std::min(C, nt - na);
        if (k < P.K - 1) {
            if (k == 0) TRY(zero_forward());
            else TRY(restore(k));
        }
        TRY(run_range<R>(c, S, 2, gf, pf, qf, na, L, st));
        const int ma = nt - na - L;
        for (int b0 = 0; b0 < L; b0 += B) {
            const int b = std::min(B, L - b0);
            TRY(run_range<R>(c, S, 3, ga, pa, qa, ma + b0, b, st));
            CK(csem::launch_td_corr<R>(seg, seg_stride, C + 1, aring, a_stride, B + 1, S, (long long)v3, nt, ma + b0, b,
                                       acc, st));
        }
    }
    // per-edge gradient divided by dV_e, then the cell mapping of csem_gradient
    CK(csem::launch_td_edges<R>(acc, -1.0 / (2.0 * c->w0 * c->dt), (long long)v3, (R *)c->d_edge, st));
    CK(csem::launch_grad_cells<R>(geo(c), (const R *)rho, (const R *)c->d_edge, wrt, c->vti != 0, (R *)grad, st));
    c->last_nrec = 0;
    return CSEM_OK;
}

template <typename R>
int time_impl(csem_ctx *c, int S, void *vol, int launches, double *ms, cudaStream_t st) {
    csem::StepParams<R> p = step_params<R>(c, true, vol);
    csem::PointParams<R> q;
    q.cE = (const R *)c->d_cE; q.step = c->d_step;
    q.nt = c->nt; q.nf = c->nf;
    q.n_rec = c->last_nrec; q.rtaps = c->d_rtaps; q.racc = c->d_racc; q.w64 = c->d_w64; q.trace = nullptr;
    q.n_itaps = 8; q.itaps = c->d_itaps; q.itap_stride = 8;
    q.n_emit = 1; q.J = 1; q.coef = c->d_ones; q.T = c->d_T;
    CK(cudaMemsetAsync(c->d_step, 0, sizeof(int), st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int cnt = std::min(c->M, c->nt);
    // the last forward run's taps (unit moments); after an adjoint run the uploaded taps
    // belong to receivers with basis-series amplitudes, so the E step is timed without them
    p.colmap = c->last_shared ? nullptr : c->d_colmap; p.colmap_stride = c->plane;
    p.tflag = c->d_tflag; p.tflag_stride = (long long)c->ny * c->nseg;
    p.inc_ntl = c->last_ntl;
    p.itaps = c->d_itaps; p.itap_stride = 8;
    p.n_emit = 1; p.J = 1; p.coef = c->d_ones; p.T = c->d_T;
    const int fkz = p.fused_kz, fzb = p.FZ_by, wlag = p.WAVE_lag;
    const int jmod = std::max(1, std::min(kChunk, c->nt - 1));   // steps within one chunk's tap increments
    if constexpr (sizeof(R) == 4) CK(csem::launch_tap_inc(p, S, kChunk, c->nt, st));
    for (int w : {0, 1, 2, 3}) {
        if (w == 1 && fkz == 0 && fzb == 0 && wlag == 0) { ms[1] = 0.0; continue; }
        auto go = [&](int j) -> cudaError_t {
            if (w == 3) return flush<R>(c, p, q, S, 0, cnt, true, c->kahan != 0, st);
            csem::StepParams<R> pp = p;
            pp.fused_kz = (w == 1) ? fkz : 0;
            pp.FZ_by = (w == 1) ? fzb : 0;
            pp.WAVE_lag = (w == 1) ? wlag : 0;
            return launch_any<R>(c, pp, q, S, j % jmod, st, w == 1 ? 5 : (w == 0 ? 1 : 4));
        };
        for (int j = 0; j < 2; ++j) CK(go(j));
        CK(cudaEventRecord(e0, st));
        for (int j = 0; j < launches; ++j) CK(go(j));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        ms[w] = (double)t / launches;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return CSEM_OK;
}

// Times the H and E kernels for every z-blocking candidate on S sources and keeps the fastest.
template <typename R>
int autotune_impl(csem_ctx *c, int S, cudaStream_t st) {
    TRY(reset_state<R>(c, S, st));
    csem::StepParams<R> p = step_params<R>(c, false, nullptr);
    csem::PointParams<R> q;
    std::memset(&q, 0, sizeof(q));
    q.step = c->d_step;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    if (c->order == 4 && sizeof(R) == 4 && c->d_cEm) {   // lean or plain fourth-order kernel per half
        for (int which : {1, 4}) {
            double best = 1e30;
            int bl = 0, bkz = 4, bmb = 4;
            for (int cand = 0; cand < 10; ++cand) {
                const int lean = cand ? 2 : 0, kz = cand ? (2 << ((cand - 1) / 3)) : 4, mb = cand ? 4 + 2 * ((cand - 1) % 3) : 4;
                p.LEAN_h = p.LEAN_e = lean;
                p.KZ_h = p.KZ_e = kz;
                p.MB_h = p.MB_e = mb;
                for (int j = 0; j < 3; ++j) CK(launch_any<R>(c, p, q, S, 0, st, which));
                CK(cudaEventRecord(e0, st));
                const int reps = 20;
                for (int j = 0; j < reps; ++j) CK(launch_any<R>(c, p, q, S, 0, st, which));
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, e0, e1));
                if (t < best) { best = t; bl = lean; bkz = kz; bmb = mb; }
            }
            if (which == 1) { c->LEAN_h = bl; c->KZ_h = bkz; c->MB_h = bmb; }
            else { c->LEAN_e = bl; c->KZ_e = bkz; c->MB_e = bmb; }
        }
        p.LEAN_h = c->LEAN_h; p.LEAN_e = c->LEAN_e;
        p.KZ_h = c->KZ_h; p.KZ_e = c->KZ_e; p.MB_h = c->MB_h; p.MB_e = c->MB_e;
    }
    if (c->order == 2) {
        const int kzs[4] = {1, 2, 4, 8};
        const int mbs[3] = {4, 6, 8};
        for (int which : {1, 4}) {
            double best = 1e30;
            int best_kz = 4, best_mb = 4, best_vec = 0;
            const int maxty = (sizeof(R) == 4) ? csem::tma_max_rows(c->pitch) : 0;
            const int ntma = maxty >= 4 ? 12 : (maxty >= 2 ? 8 : (maxty >= 1 ? 4 : 0));
            const int nlean = (sizeof(R) == 4 && c->d_psiL) ? 15 : 0;
            const int ncand = (sizeof(R) == 4) ? 20 + ntma + nlean : 12;   // 12 scalar, 8 four-cell, staged, lean
            int best_tma = 0, best_lean = 0;
            for (int cand = 0; cand < ncand; ++cand) {
                const int lc = cand - 20 - ntma;
                const int lean = (lc >= 0) ? (lc < 6 ? 1 : 2) : 0;                            // cells per thread 1, 2
                const int vec = (cand >= 12 && cand < 20) ? 1 : 0;
                const int tma = (cand >= 20 && !lean) ? (1 << ((cand - 20) / 4)) : 0;          // rows per block 1, 2, 4
                const int tkz[4] = {2, 4, 8, 16}, lkz[3] = {1, 2, 4};
                const int kz = lean ? lkz[lc % 3] : (tma ? tkz[(cand - 20) % 4] : kzs[cand % 4]);
                const int lmb[3] = {6, 8, 4};   // 1 cell: 6, 8; 2 cells: 6, 8, 4 blocks of 128 threads per SM
                const int mb = lean ? lmb[(lc % (lc < 6 ? 6 : 9)) / 3] : (tma ? 4 : (vec ? mbs[(cand - 12) / 4] : mbs[cand / 4]));
                p.KZ_h = p.KZ_e = kz;
                p.MB_h = p.MB_e = mb;
                p.VEC_h = p.VEC_e = vec;
                p.TMA_h = p.TMA_e = tma;
                p.LEAN_h = p.LEAN_e = lean;
                for (int j = 0; j < 3; ++j) CK(csem::launch_step<R>(p, q, S, 0, st, which));
                CK(cudaEventRecord(e0, st));
                const int reps = 20;
                for (int j = 0; j < reps; ++j) CK(csem::launch_step<R>(p, q, S, 0, st, which));
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, e0, e1));
                if (t < best) { best = t; best_kz = kz; best_mb = mb; best_vec = vec; best_tma = tma; best_lean = lean; }
            }
            if (which == 1) { c->KZ_h = best_kz; c->MB_h = best_mb; c->VEC_h = best_vec; c->TMA_h = best_tma; c->LEAN_h = best_lean; }
            else { c->KZ_e = best_kz; c->MB_e = best_mb; c->VEC_e = best_vec; c->TMA_e = best_tma; c->LEAN_e = best_lean; }
        }
        // fused H+E steps against the best split pair: the tiled kernel (kz 4, 8, 16) and,
        // for FP32 with nx even, the one-pass kernel (rows per block and resident blocks
        // (4, 4), (4, 6), (8, 2), (8, 3), z blocks of 8, 16, 32, 64 planes), the
        // warp-specialised one, and the wave-ordered step (both lean halves in one launch)
        {
            p.KZ_h = c->KZ_h; p.KZ_e = c->KZ_e; p.MB_h = c->MB_h; p.MB_e = c->MB_e;
            p.VEC_h = c->VEC_h; p.VEC_e = c->VEC_e;
            p.TMA_h = c->TMA_h; p.TMA_e = c->TMA_e;
            p.LEAN_h = c->LEAN_h; p.LEAN_e = c->LEAN_e;
            struct Cand { int f, by, mb, kz, ws, lag; };
            std::vector<Cand> cands = {{0, 0, 4, 16, 0, 0}, {4, 0, 4, 16, 0, 0}, {8, 0, 4, 16, 0, 0}, {16, 0, 4, 16, 0, 0}};
            if (sizeof(R) == 4 && c->d_q && c->nx % 2 == 0) {
                const int bm[4][2] = {{4, 4}, {4, 6}, {8, 2}, {8, 3}};
                for (const auto &b : bm)
                    for (int kz : {8, 16, 32, 64}) cands.push_back({0, b[0], b[1], kz, 0, 0});
                if (c->d_cEm && c->d_psi) {        // the warp-specialised fused step
                    const int wm[5][2] = {{4, 2}, {4, 3}, {6, 2}, {8, 1}, {8, 2}};
                    for (const auto &b : wm)
                        for (int kz : {8, 16, 32, 64}) cands.push_back({0, b[0], b[1], kz, 1, 0});
                }
                // the wave-ordered step: E lagging H by 1 to 4 z blocks of 2 or 4 planes, 6 or 8 blocks/SM
                if constexpr (sizeof(R) == 4) {
                    for (int kz : {2, 4})
                        for (int mb : {6, 8})
                            if (csem::wave_supported(p, kz, mb))
                                for (int lag : {1, 2, 3, 4}) cands.push_back({0, 0, mb, kz, 0, lag});
                }
            }
            auto time_cand = [&](const Cand &cd, float *t) -> int {
                p.fused_kz = cd.f;
                p.FZ_by = cd.by; p.FZ_mb = cd.mb; p.FZ_kz = cd.kz; p.FZ_ws = cd.ws;
                p.WAVE_lag = cd.lag; p.WAVE_kz = cd.lag ? cd.kz : 4; p.WAVE_mb = cd.lag ? cd.mb : 8;
                for (int j = 0; j < 3; ++j) CK(csem::launch_step<R>(p, q, S, 0, st, 5));
                CK(cudaEventRecord(e0, st));
                const int reps = 20;
                for (int j = 0; j < reps; ++j) CK(csem::launch_step<R>(p, q, S, 0, st, 5));
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                CK(cudaEventElapsedTime(t, e0, e1));
                return CSEM_OK;
            };
            // first pass: the fastest fused candidate; then the split pair and that candidate
            // are timed again, alternately, three times each, and the lower median wins, so the
            // choice does not hang on one measurement (or on which candidate ran first)
            double best = 1e30;
            Cand bc = cands[0];
            for (size_t u = 1; u < cands.size(); ++u) {
                float t = 0.f;
                TRY(time_cand(cands[u], &t));
                if (t < best) { best = t; bc = cands[u]; }
            }
            float ts[3], tf[3];
            for (int r = 0; r < 3; ++r) {
                TRY(time_cand(cands[0], &ts[r]));
                TRY(time_cand(bc, &tf[r]));
            }
            std::sort(ts, ts + 3);
            std::sort(tf, tf + 3);
            if (!(tf[1] < ts[1])) bc = cands[0];
            c->fused_kz = bc.f;
            c->FZ_by = bc.by; c->FZ_mb = bc.mb; c->FZ_kz = bc.kz; c->FZ_ws = bc.ws;
            c->WAVE_lag = bc.lag; c->WAVE_kz = bc.lag ? bc.kz : 4; c->WAVE_mb = bc.lag ? bc.mb : 8;
            p.fused_kz = 0;
            p.FZ_by = 0;
            p.WAVE_lag = 0;
        }
    }
    // transform flush: register or bulk copy (FP32), 16 or 32 snapshots, after
    // its block or overlapping the next one (when the ring has room); each
    // candidate is timed over 2 kChunk steps with its flushes, from step kChunk on
    if (c->nt >= 4 * kChunk) {
        typedef typename C2<R>::T R2;
        R2 *vol_tmp = nullptr;
        const size_t vb = (size_t)S * 3 * c->nf * c->vol * sizeof(R2);
        if (cudaMallocAsync((void **)&vol_tmp, vb, st) == cudaSuccess) {
            CK(cudaMemsetAsync(vol_tmp, 0, vb, st));
            p.acc = vol_tmp;
            p.comp = c->kahan ? (R2 *)c->d_comp : nullptr;
            p.fused_kz = c->fused_kz;
            p.FZ_by = c->FZ_by; p.FZ_mb = c->FZ_mb; p.FZ_kz = c->FZ_kz; p.FZ_ws = c->FZ_ws;
            p.WAVE_lag = c->WAVE_lag; p.WAVE_kz = c->WAVE_kz; p.WAVE_mb = c->WAVE_mb;
            const bool kahan = c->kahan != 0;
            double best = 1e30;
            int bm = 0, bM = 16;
            for (int mode = 0; mode < 4; ++mode)
                for (int m : {16, 32, 64, 128}) {
                    if ((mode & 1) && sizeof(R) != 4) continue;
                    if (((mode & 2) ? 2 * m : m) + 1 > c->nslot) continue;
                    c->flush_mode = mode;
                    c->M = m;
                    CK(cudaMemsetAsync(c->d_step, 0, sizeof(int), st));
                    CK(csem::launch_advance(c->d_step, kChunk, st));
                    CK(emit_steps<R>(c, S, true, kahan, p, q, kChunk, false, true, st));
                    CK(cudaEventRecord(e0, st));
                    CK(emit_steps<R>(c, S, true, kahan, p, q, 2 * kChunk, false, true, st));
                    CK(cudaEventRecord(e1, st));
                    CK(cudaEventSynchronize(e1));
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, e0, e1));
                    if (t < best) { best = t; bm = mode; bM = m; }
                }
            c->flush_mode = bm;
            c->M = bM;
            CK(cudaMemsetAsync(c->d_step, 0, sizeof(int), st));
            cudaFreeAsync(vol_tmp, st);
        } else {
            cudaGetLastError();
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return CSEM_OK;
}

void free_ctx(csem_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    void *ptrs[] = {c->d_wave, c->d_q, c->d_tabG, c->d_ho, c->d_tabL, c->d_psiL, c->d_cEm, c->d_inc, c->d_tapk, c->d_tab, c->d_h, c->d_cE, c->d_H, c->d_H2, c->d_ering, c->d_psi, c->d_comp, c->d_edge, c->d_wR, c->d_w64,
                    c->d_alpha, c->d_racc, c->d_coef, c->d_T, c->d_ones, c->d_rtaps, c->d_itaps, c->d_colmap, c->d_tflag, c->d_cpos, c->d_cval, c->d_step, c->d_bad};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (void *p : {(void *)c->d_rprev, (void *)c->d_rfin, (void *)c->d_es, c->d_vprev, (void *)c->d_vstats})
        if (p) cudaFree(p);
    if (c->h_es) cudaFreeHost(c->h_es);
    for (int k = 0; k < kEsDepth; ++k)
        if (c->es_ev[k]) cudaEventDestroy(c->es_ev[k]);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->side) cudaStreamDestroy(c->side);
    for (int k = 0; k < kMaxSide; ++k) {
        if (c->ev_fork[k]) cudaEventDestroy(c->ev_fork[k]);
        if (c->ev_done[k]) cudaEventDestroy(c->ev_done[k]);
    }
    delete c;
}

}  // namespace

extern "C" {

const char *csem_last_error(void) { return g_err.c_str(); }

int csem_create(csem_ctx **out, const csem_grid *g, const csem_opts *o) {
    if (!out || !g || !o) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (g->npml < 0 || g->nx < 2 * g->npml + 2 || g->ny < 2 * g->npml + 2 || g->nz < 2 * g->npml + 2)
        return fail(CSEM_ERR_INVALID_ARG, "grid too small for its CPML");
    if (!g->xn || !g->yn || !g->zn) return fail(CSEM_ERR_INVALID_ARG, "NULL node coordinates");
    if (o->precision != 32 && o->precision != 64) return fail(CSEM_ERR_INVALID_ARG, "precision must be 32 or 64");
    if (o->n_freq < 1 || o->n_freq > csem::kMaxFreq || !o->freqs)
        return fail(CSEM_ERR_INVALID_ARG, "n_freq must be in 1..8");
    if (!(o->f0 > 0.0) || !(o->rho_max > 0.0)) return fail(CSEM_ERR_INVALID_ARG, "f0 and rho_max must be > 0");
    if (o->anisotropy != 0 && o->anisotropy != 1) return fail(CSEM_ERR_INVALID_ARG, "anisotropy must be 0 or 1");
    if (o->order != 0 && o->order != 2 && o->order != 4) return fail(CSEM_ERR_INVALID_ARG, "order must be 2 or 4");
    if (o->max_src < 1 || o->max_rec < 0 || o->max_src > 65535)
        return fail(CSEM_ERR_INVALID_ARG, "max_src must be >= 1, max_rec >= 0");
    for (int f = 0; f < o->n_freq; ++f)
        if (!(o->freqs[f] > 0.0) || !std::isfinite(o->freqs[f])) return fail(CSEM_ERR_INVALID_ARG, "bad frequency");

    csem_ctx *c = new csem_ctx();
    cudaGetDevice(&c->device);
    c->nx = g->nx; c->ny = g->ny; c->nz = g->nz; c->npml = g->npml;
    c->NX = c->nx + 1; c->NY = c->ny + 1; c->NZ = c->nz + 1;
    c->pitch = (c->NX + 7) / 8 * 8;
    c->plane = (long long)c->pitch * c->NY;
    c->vol = c->plane * c->NZ;
    const int ns[3] = {c->nx, c->ny, c->nz};
    const double *xs[3] = {g->xn, g->yn, g->zn};
    double inv2max[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        Axis &A = c->ax[a];
        A.n = ns[a];
        A.x.assign(xs[a], xs[a] + A.n + 1);
        A.h.resize(A.n);
        A.ht.resize(A.n + 1);
        for (int i = 0; i < A.n; ++i) {
            A.h[i] = A.x[i + 1] - A.x[i];
            if (!(A.h[i] > 0.0) || !std::isfinite(A.h[i])) {
                delete c;
                return fail(CSEM_ERR_INVALID_ARG, "node coordinates must be finite and strictly increasing");
            }
            inv2max[a] = std::max(inv2max[a], 1.0 / (A.h[i] * A.h[i]));
        }
        A.ht[0] = 0.5 * A.h[0];
        A.ht[A.n] = 0.5 * A.h[A.n - 1];
        for (int i = 1; i < A.n; ++i) A.ht[i] = 0.5 * (A.h[i - 1] + A.h[i]);
    }
    c->f0 = o->f0;
    c->w0 = 2.0 * M_PI * o->f0;
    c->rho_max = o->rho_max;
    c->safety = o->cfl_safety > 0.0 ? o->cfl_safety : 0.99;
    // fictitious speed v = 1/sqrt(mu0 eps), eps = sigma/(2 w0)  (Eq. 2)
    const double vmax = std::sqrt(2.0 * c->w0 * c->rho_max / kMu0);
    c->order = o->order == 4 ? 4 : 2;
    double dt_lim = 1.0 / (vmax * std::sqrt(inv2max[0] + inv2max[1] + inv2max[2]));
    if (c->order == 4) {
        // leap-frog limit 2 / (v sqrt(sum over axes of the largest symbol squared)); the
        // cells form a tensor product, so the largest sum is the sum of the per-axis maxima
        double s2 = 0.0;
        for (int a = 0; a < 3; ++a) { const double sm = ho_axis(c->ax[a]); s2 += sm * sm; }
        dt_lim = 2.0 / (vmax * std::sqrt(s2));
    }
    if (o->dt > 0.0) {
        if (o->dt > dt_lim * (1.0 + 1e-12)) {
            delete c;
            return fail(CSEM_ERR_CFL, "dt above the CFL limit " + std::to_string(dt_lim));
        }
        c->dt = o->dt;
    } else {
        c->dt = c->safety * dt_lim;
    }
    c->nf = o->n_freq;
    c->freqs.assign(o->freqs, o->freqs + c->nf);
    c->a.resize(c->nf);
    c->kf.resize(c->nf);
    double amin = 1e300;
    for (int f = 0; f < c->nf; ++f) {
        const double w = 2.0 * M_PI * c->freqs[f];
        c->a[f] = std::sqrt(w * c->w0);
        amin = std::min(amin, c->a[f]);
        // k = sqrt(-i w / (2 w0)) on the principal branch = (1 - i)/2 sqrt(w / w0)  (Eq. 3)
        c->kf[f] = std::sqrt(std::complex<double>(0.0, -w / (2.0 * c->w0)));
    }
    c->nt = o->nt > 0 ? o->nt : (int)std::ceil(kDecaySpan / (amin * c->dt));
    c->precision = o->precision;
    c->kahan = (o->precision == 32 && o->kahan) ? 1 : 0;
    c->max_src = o->max_src;
    c->max_rec = o->max_rec;
    c->vti = o->anisotropy;
    c->rsize = (c->precision == 32) ? 4 : 8;
    for (int a = 0; a < 3; ++a) cpml_axis(c->ax[a], c->npml, c->dt, vmax, c->f0);
    const int np2 = 2 * c->npml;
    auto pad8 = [](long long v) { return (v + 7) / 8 * 8; };   // keeps every slab array 32-byte aligned
    c->sx = pad8((long long)c->NZ * c->NY * np2);
    c->sy = pad8((long long)c->NZ * np2 * c->pitch);
    c->sz = pad8((long long)np2 * c->NY * c->pitch);
    c->psi_stride = c->order == 4 ? 12 * c->vol : 6 * (c->sx + c->sy + c->sz);
    c->wavelet.assign(c->nt, 0.0);
    c->wavelet[0] = 1.0 / c->dt;

    // E ring: 2M + 1 slots for an M-snapshot flush that overlaps the next block,
    // M + 1 otherwise (M = 16, 32, 64): 129, 65, 33 or 17 slots, the largest that
    // fits in 85 % of the free memory beside the rest of the per-source state and
    // the transform volumes a gradient holds (forward and adjoint, and the Kahan
    // terms)
    {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const double S = c->max_src, V = (double)c->vol, r = (double)c->rsize;
        const double slot = S * 3 * V * r;
        const double vols = S * 3 * c->nf * V * 2 * r * (c->kahan ? 3 : 2);
        const double rest = S * (6 * V * r + (double)c->psi_stride * r + (c->precision == 32 ? 12 * V * 4 : 0)) +
                            6 * V * r;
        c->nslot = 17;
        for (int ns : {129, 65, 33})
            if ((o->ring_slots <= 0 || ns <= o->ring_slots) && ns * slot + vols + rest < 0.85 * (double)free_b) {
                c->nslot = ns;
                break;
            }
        c->M = 16;
    }
    int rc = CSEM_OK;
    auto step = [&](int r) { if (rc == CSEM_OK) rc = r; };
    if (c->precision == 32) step(upload_tables<float>(c)); else step(upload_tables<double>(c));
    const size_t R = c->rsize, C2s = 2 * R;
    const int S = c->max_src, NR = std::max(c->max_rec, 1);
    step(dalloc(c, &c->d_h, (size_t)(c->nx + c->ny + c->nz) * sizeof(double)));
    step(dalloc(c, &c->d_cE, 3 * (size_t)c->vol * R));
    step(dalloc(c, &c->d_edge, 3 * (size_t)c->vol * R));
    step(dalloc(c, &c->d_H, (size_t)S * 3 * c->vol * R));
    step(dalloc(c, &c->d_H2, (size_t)S * 3 * c->vol * R));
    step(dalloc(c, &c->d_ering, (size_t)S * c->nslot * 3 * c->vol * R));
    step(dalloc(c, &c->d_psi, (size_t)S * c->psi_stride * R));
    if (c->kahan) step(dalloc(c, &c->d_comp, (size_t)S * 3 * c->nf * c->vol * C2s));
    step(dalloc(c, &c->d_alpha, 3 * (size_t)c->nf * sizeof(double2)));
    step(dalloc(c, &c->d_racc, (size_t)S * NR * c->nf * sizeof(double2)));
    step(dalloc(c, &c->d_coef, (size_t)S * NR * 2 * c->nf * sizeof(double)));
    step(dalloc(c, &c->d_T, (size_t)c->nt * sizeof(double)));
    step(dalloc(c, &c->d_ones, (size_t)S * sizeof(double)));
    step(dalloc(c, &c->d_rtaps, (size_t)NR * 8 * sizeof(Tap)));
    step(dalloc(c, &c->d_itaps, (size_t)std::max(S, NR) * 8 * sizeof(Tap)));
    step(dalloc(c, &c->d_colmap, (size_t)S * c->plane * sizeof(int2)));
    c->nseg = (c->nx + 31) / 32;
    step(dalloc(c, &c->d_tflag, (size_t)std::max(S, NR) * c->ny * c->nseg));
    step(dalloc(c, &c->d_cpos, (size_t)std::max(S, NR) * 8 * sizeof(long long)));
    step(dalloc(c, &c->d_cval, (size_t)std::max(S, NR) * 8 * sizeof(int2)));
    step(dalloc(c, &c->d_step, sizeof(int)));
    step(dalloc(c, &c->d_bad, sizeof(int)));
    // lean FP32 kernels: CPML memory as 12 volume arrays per source and the masked dt/eps
    if (rc == CSEM_OK && c->order == 4) {
        std::vector<double> t;
        for (int a = 0; a < 3; ++a) {
            t.insert(t.end(), c->ax[a].wh.begin(), c->ax[a].wh.end());
            t.insert(t.end(), c->ax[a].wn.begin(), c->ax[a].wn.end());
        }
        if (c->precision == 32) {
            std::vector<float> tf(t.begin(), t.end());
            step(dalloc(c, (float **)&c->d_ho, tf.size() * sizeof(float)));
            if (rc == CSEM_OK && cudaMemcpy(c->d_ho, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
                rc = fail(CSEM_ERR_CUDA, "context initialisation failed");
        } else {
            step(dalloc(c, (double **)&c->d_ho, t.size() * sizeof(double)));
            if (rc == CSEM_OK && cudaMemcpy(c->d_ho, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
                rc = fail(CSEM_ERR_CUDA, "context initialisation failed");
        }
    }
    // FP32, nx even: tap increments and padded tables (and for the fourth order the masked
    // dt/eps of its lean kernels); second order also the fused one-pass step's per-cell
    // material and widths, and for the lean split kernels (nx a multiple of 4) the CPML
    // memory in 12 volume arrays per source, kept when it fits
    if (rc == CSEM_OK && c->precision == 32 && c->nx % 2 == 0) {
        step(dalloc(c, &c->d_inc, (size_t)kChunk * S * std::max(8, NR * 8) * sizeof(float)));
        step(dalloc(c, &c->d_tapk, (size_t)std::max(S, NR) * 8 * sizeof(int)));
        step(upload_lean_tables(c));
        if (c->order == 4) {                 // lean fourth-order kernels: masked dt/eps
            step(dalloc(c, &c->d_cEm, 3 * (size_t)c->vol * sizeof(float)));
            if (rc == CSEM_OK && cudaMemset(c->d_cEm, 0, 3 * (size_t)c->vol * sizeof(float)) != cudaSuccess)
                rc = fail(CSEM_ERR_CUDA, "context initialisation failed");
        }
    }
    if (rc == CSEM_OK && c->order == 2 && c->precision == 32 && c->nx % 2 == 0) {
        if (rc == CSEM_OK) step(upload_geo_tables(c));
        const size_t qb = (size_t)(c->vti ? 2 : 1) * c->vol * sizeof(float);
        step(dalloc(c, &c->d_q, qb));
        // finite, positive values (bytes 0x3f: 0.747f) until a run sets the model, so the
        // autotuner times the fused step on finite arithmetic
        if (rc == CSEM_OK && cudaMemset(c->d_q, 0x3f, qb) != cudaSuccess)
            rc = fail(CSEM_ERR_CUDA, "context initialisation failed");
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const double need = ((double)S * 12 + 3) * c->vol * sizeof(float);
        if (rc == CSEM_OK && c->nx % 4 == 0 && need < 0.25 * (double)free_b) {
            step(dalloc(c, &c->d_psiL, (size_t)S * 12 * c->vol * sizeof(float)));
            step(dalloc(c, &c->d_cEm, 3 * (size_t)c->vol * sizeof(float)));
            step(dalloc(c, &c->d_wave, (2 + csem::kMaxWaveChunks) * sizeof(unsigned)));
            if (rc == CSEM_OK && (cudaMemset(c->d_cEm, 0, 3 * (size_t)c->vol * sizeof(float)) != cudaSuccess ||
                                  cudaMemset(c->d_wave, 0, (2 + csem::kMaxWaveChunks) * sizeof(unsigned)) != cudaSuccess))
                rc = fail(CSEM_ERR_CUDA, "context initialisation failed");
        }
    }
    if (rc != CSEM_OK) { free_ctx(c); return rc; }
    std::vector<double> hcat;
    for (int a = 0; a < 3; ++a) hcat.insert(hcat.end(), c->ax[a].h.begin(), c->ax[a].h.end());
    std::vector<double> ones((size_t)S, 1.0);
    if (cudaMemcpy(c->d_h, hcat.data(), hcat.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_ones, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_bad, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_cE, 0, 3 * (size_t)c->vol * c->rsize) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) {
        free_ctx(c);
        return fail(CSEM_ERR_CUDA, "context initialisation failed");
    }
    for (int k = 0; k < kMaxSide; ++k)
        if (cudaEventCreateWithFlags(&c->ev_fork[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming) != cudaSuccess) {
            free_ctx(c);
            return fail(CSEM_ERR_CUDA, "context initialisation failed");
        }
    rc = update_wavelet(c);
    if (rc != CSEM_OK) { free_ctx(c); return rc; }
    {
        cudaError_t e1 = csem::prepare_bulk_flush(), e2 = csem::prepare_fused_all(), e3 = csem::prepare_tma();
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            cudaGetLastError();
            free_ctx(c);
            return fail(CSEM_ERR_CUDA, std::string("cannot configure shared memory of the ") +
                                           (e1 != cudaSuccess ? "bulk-copy flush" : e2 != cudaSuccess ? "fused step" : "staged step") +
                                           " kernels");
        }
    }
    *out = c;
    return CSEM_OK;
}

void csem_destroy(csem_ctx *c) { free_ctx(c); }

int csem_get_info(const csem_ctx *c, csem_info *info) {
    if (!c || !info) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    info->nx = c->nx; info->ny = c->ny; info->nz = c->nz; info->npml = c->npml;
    info->pitch = c->pitch; info->vol_elems = c->vol; info->dt = c->dt; info->nt = c->nt;
    info->order = c->order;
    info->precision = c->precision; info->kahan = c->kahan; info->n_freq = c->nf;
    info->max_src = c->max_src; info->max_rec = c->max_rec; info->workspace_bytes = c->bytes;
    info->transform_block = c->M;
    info->anisotropy = c->vti;
    return CSEM_OK;
}

int csem_set_wavelet(csem_ctx *c, const double *w) {
    if (!c) return fail(CSEM_ERR_INVALID_ARG, "NULL context");
    CK(cudaDeviceSynchronize());
    if (w) c->wavelet.assign(w, w + c->nt);
    else { c->wavelet.assign(c->nt, 0.0); c->wavelet[0] = 1.0 / c->dt; }
    return update_wavelet(c);
}

int csem_set_copy_fault(csem_ctx *c, int extra_bytes) {
    if (!c || extra_bytes < 0 || extra_bytes > 4096 || extra_bytes % 16 != 0)
        return fail(CSEM_ERR_INVALID_ARG, "extra_bytes must be a multiple of 16 in 0..4096");
    CK(cudaDeviceSynchronize());
    c->fault_tx = extra_bytes;
    return CSEM_OK;
}

int csem_set_trace(csem_ctx *c, double *trace_dev) {
    if (!c) return fail(CSEM_ERR_INVALID_ARG, "NULL context");
    c->d_trace = trace_dev;
    return CSEM_OK;
}

int csem_check(csem_ctx *c, void *stream) {
    if (!c) return fail(CSEM_ERR_INVALID_ARG, "NULL context");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    int bad = 0;
    CK(cudaMemcpy(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(c->d_bad, 0, sizeof(int)));
    if (bad & (csem::kErrFlushWait | csem::kErrStagedWait | csem::kErrOnepassWait | csem::kErrWaveWait)) {
        std::string who;
        auto add = [&](const char *w) { who += (who.empty() ? "" : " and ") + std::string(w); };
        if (bad & csem::kErrFlushWait) add("a bulk-copy transform flush");
        if (bad & csem::kErrStagedWait) add("a row-staged H/E step kernel");
        if (bad & csem::kErrOnepassWait) add("a fused step kernel (one-pass or warp-specialised)");
        if (bad & csem::kErrWaveWait) add("an E tile of the wave-ordered step");
        return fail(CSEM_ERR_TIMEOUT, who + " gave up a bounded wait (the results of that run are not valid)");
    }
    if (bad & csem::kErrNonfinite) return fail(CSEM_ERR_NONFINITE, "a resistivity was non-positive or non-finite");
    return CSEM_OK;
}

int csem_fwd_model(csem_ctx *c, const void *rho_dev, const csem_points *src, const csem_points *rec,
                   double *d_syn_dev, void *Evol_dev, void *stream) {
    if (!c || !rho_dev) return fail(CSEM_ERR_INVALID_ARG, "NULL context or model");
    TRY(check_points(src, c->max_src, "sources", false));
    TRY(check_points(rec, c->max_rec, "receivers", true));
    if (rec->n > 0 && !d_syn_dev) return fail(CSEM_ERR_INVALID_ARG, "d_syn_dev is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    return c->precision == 32 ? fwd_impl<float>(c, rho_dev, src, rec, d_syn_dev, Evol_dev, st)
                              : fwd_impl<double>(c, rho_dev, src, rec, d_syn_dev, Evol_dev, st);
}

int csem_adjoint_model(csem_ctx *c, const void *rho_dev, const csem_points *rec, int n_src, const double *resid_dev,
                       const double *basis_dev, void *Vvol_dev, void *stream) {
    if (!c || !rho_dev || !resid_dev || !basis_dev || !Vvol_dev) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    TRY(check_points(rec, c->max_rec, "receivers", false));
    if (n_src < 1 || n_src > c->max_src) return fail(CSEM_ERR_INVALID_ARG, "n_src out of range");
    cudaStream_t st = (cudaStream_t)stream;
    return c->precision == 32 ? adj_impl<float>(c, rho_dev, rec, n_src, resid_dev, basis_dev, Vvol_dev, st)
                              : adj_impl<double>(c, rho_dev, rec, n_src, resid_dev, basis_dev, Vvol_dev, st);
}

int csem_gradient(csem_ctx *c, const void *rho_dev, const void *Evol_dev, const void *Vvol_dev, int n_src, int wrt,
                  void *grad_dev, void *stream) {
    if (!c || !rho_dev || !Evol_dev || !Vvol_dev || !grad_dev) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    if (n_src < 1 || (wrt != 0 && wrt != 1)) return fail(CSEM_ERR_INVALID_ARG, "bad n_src or wrt");
    cudaStream_t st = (cudaStream_t)stream;
    if (c->precision == 32)
        CK(csem::launch_gradient<float>(geo(c), (const float *)rho_dev, (const float2 *)Evol_dev,
                                        (const float2 *)Vvol_dev, n_src, c->nf, wrt, c->vti != 0, (float *)c->d_edge,
                                        (float *)grad_dev, st));
    else
        CK(csem::launch_gradient<double>(geo(c), (const double *)rho_dev, (const double2 *)Evol_dev,
                                         (const double2 *)Vvol_dev, n_src, c->nf, wrt, c->vti != 0, (double *)c->d_edge,
                                         (double *)grad_dev, st));
    return CSEM_OK;
}

int csem_td_plan(const csem_ctx *c, int n_src, int n_rec, long long budget_bytes, int *segment_out,
                 long long *bytes_out) {
    if (!c || !segment_out || !bytes_out) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    if (n_src < 1 || n_src > c->max_src || n_rec < 1 || n_rec > c->max_rec)
        return fail(CSEM_ERR_INVALID_ARG, "n_src or n_rec out of range");
    TdPlan P;
    TRY(td_plan(c, n_src, n_rec, *segment_out > 0 ? *segment_out : 0, budget_bytes, &P));
    *segment_out = P.C;
    *bytes_out = (long long)P.total;
    return CSEM_OK;
}

int csem_gradient_td(csem_ctx *c, const void *rho_dev, const csem_points *src, const csem_points *rec,
                     const double *resid_dev, int segment, int wrt, void *grad_dev, void *work_dev,
                     long long work_bytes, void *stream) {
    if (!c || !rho_dev || !resid_dev || !grad_dev || !work_dev) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    TRY(check_points(src, c->max_src, "sources", false));
    TRY(check_points(rec, c->max_rec, "receivers", false));
    if (segment < 2 || (wrt != 0 && wrt != 1)) return fail(CSEM_ERR_INVALID_ARG, "bad segment or wrt");
    cudaStream_t st = (cudaStream_t)stream;
    return c->precision == 32
               ? td_impl<float>(c, rho_dev, src, rec, resid_dev, segment, wrt, grad_dev, work_dev, work_bytes, st)
               : td_impl<double>(c, rho_dev, src, rec, resid_dev, segment, wrt, grad_dev, work_dev, work_bytes, st);
}

namespace {
// The device state {ended, steps}, its pinned host copies and events, shared by both early ends.
int es_state(csem_ctx *c) {
    if (!c->d_es) TRY(dalloc(c, &c->d_es, 2 * sizeof(int)));
    if (!c->h_es) CK(cudaHostAlloc((void **)&c->h_es, kEsDepth * sizeof(int), cudaHostAllocDefault));
    for (int k = 0; k < kEsDepth; ++k)
        if (!c->es_ev[k]) CK(cudaEventCreateWithFlags(&c->es_ev[k], cudaEventDisableTiming));
    return CSEM_OK;
}
}  // namespace

int csem_set_early_stop(csem_ctx *c, double tol) {
    if (!c || !(tol >= 0.0) || !std::isfinite(tol)) return fail(CSEM_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (tol > 0.0) {
        TRY(es_state(c));
        if (!c->d_rprev) {
            const size_t nb = (size_t)c->max_src * std::max(c->max_rec, 1) * c->nf * sizeof(double2);
            TRY(dalloc(c, &c->d_rprev, nb));
            TRY(dalloc(c, &c->d_rfin, nb));
        }
    }
    c->es_tol = tol;
    return CSEM_OK;
}

int csem_set_early_stop_volumes(csem_ctx *c, double tol, double floor_frac) {
    if (!c || !(tol >= 0.0) || !std::isfinite(tol)) return fail(CSEM_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (!(floor_frac >= 0.0) || !(floor_frac <= 1.0)) return fail(CSEM_ERR_INVALID_ARG, "floor_frac must be in [0, 1]");
    if (tol > 0.0) {
        TRY(es_state(c));
        if (!c->d_vprev) {
            TRY(dalloc(c, (char **)&c->d_vprev, (size_t)c->max_src * 3 * c->nf * c->vol * 2 * c->rsize));
            TRY(dalloc(c, &c->d_vstats, 3 * (size_t)c->nf * sizeof(unsigned)));
        }
    }
    c->es_vol_tol = tol;
    c->es_vol_floor = floor_frac;
    return CSEM_OK;
}

int csem_last_run_steps(csem_ctx *c, void *stream, int *steps) {
    if (!c || !steps) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    if (!c->last_es) { *steps = c->nt; return CSEM_OK; }
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    int st[2] = {0, 0};
    CK(cudaMemcpy(st, c->d_es, sizeof(st), cudaMemcpyDeviceToHost));
    *steps = st[0] ? st[1] : c->nt;
    return CSEM_OK;
}

long long csem_launch_count(void) { return csem::g_launches.load(); }

int csem_set_launch(csem_ctx *c, const int *cfg) {
    if (!c || !cfg) return fail(CSEM_ERR_INVALID_ARG, "NULL argument");
    const int kzh = cfg[0], mbh = cfg[1], kze = cfg[2], mbe = cfg[3], fm = cfg[5], M = cfg[6];
    // cfg[4] >= 10000: the fused one-pass step, 10000 + planes * 100 + rows * 10 + blocks;
    // cfg[4] >= 30000: the warp-specialised fused step, 30000 + the same code;
    // cfg[4] >= 50000: the wave-ordered step, 50000 + lag * 100 + planes * 10 + blocks
    const int wv = cfg[4] >= 50000 ? cfg[4] - 50000 : 0;
    const int wv_lag = wv / 100, wv_kz = (wv / 10) % 10, wv_mb = wv % 10;
    if (wv) {
        csem::StepParams<float> tp{};
        tp.nx = c->nx; tp.nz = c->nz; tp.psiL = c->d_psiL; tp.cEm = c->d_cEm; tp.wave = c->d_wave;
        tp.lx.ih_n = c->d_tabL ? (const float *)c->d_tabL : nullptr; tp.lzero = tp.lx.ih_n;
        if (c->precision != 32 || c->order != 2 || wv_lag < 1 || !csem::wave_supported(tp, wv_kz, wv_mb))
            return fail(CSEM_ERR_INVALID_ARG, "wave-ordered step: FP32, second order, nx a multiple of 4, lag >= 1, 2 or 4 planes, 6 or 8 blocks/SM");
    }
    const int ws = (!wv && cfg[4] >= 30000) ? 1 : 0;
    const int fz = (!wv && cfg[4] >= 10000) ? cfg[4] - (ws ? 30000 : 10000) : 0, fkz = (fz || wv) ? 0 : cfg[4];
    const int fz_kz = fz / 100, fz_by = (fz / 10) % 10, fz_mb = fz % 10;
    if (fz && !ws && (c->precision != 32 || c->order != 2 || !c->d_q || c->nx % 2 != 0 || !csem::fz_supported(fz_by, fz_mb, fz_kz)))
        return fail(CSEM_ERR_INVALID_ARG, "fused one-pass step: FP32, second order, nx even, rows/blocks (4,4), (4,6), (8,2) or (8,3), 2-99 planes");
    if (ws && (c->precision != 32 || c->order != 2 || !c->d_q || !c->d_cEm || !c->d_psi || c->nx % 2 != 0 ||
               !csem::ws_supported(fz_by, fz_mb, fz_kz)))
        return fail(CSEM_ERR_INVALID_ARG, "warp-specialised fused step: FP32, second order, nx a multiple of 4, rows/blocks (4,2), (4,3), (6,2), (8,1) or (8,2), 2-99 planes");
    const int vh = cfg[7], ve = cfg[8], th = cfg[9], te = cfg[10], lh = cfg[11], le = cfg[12];
    if (c->order == 4) {   // fourth order: its own kernels, the lean FP32 ones (2 cells) per half
        if (fkz || fz || vh || ve || th || te)
            return fail(CSEM_ERR_INVALID_ARG, "a fourth-order context runs its own H and E kernels only");
        auto ok = [&](int l, int kz, int mb) { return l == 0 || (l == 2 && csem::ho4_supported(kz, mb)); };
        if ((lh || le) && (c->precision != 32 || !c->d_cEm || !ok(lh, kzh, mbh) || !ok(le, kze, mbe)))
            return fail(CSEM_ERR_INVALID_ARG, "lean fourth-order kernels: FP32, nx even, 2 cells, 2/4/8 planes, 4/6/8 blocks/SM");
        if (fm < 0 || fm > 3 || ((fm & 1) && c->precision != 32) || !(M == 16 || M == 32 || M == 64 || M == 128) ||
            ((fm & 2) ? 2 * M : M) + 1 > c->nslot)
            return fail(CSEM_ERR_INVALID_ARG, "launch configuration not supported by this context");
        CK(cudaDeviceSynchronize());
        c->KZ_h = lh ? kzh : 4; c->MB_h = lh ? mbh : 4; c->KZ_e = le ? kze : 4; c->MB_e = le ? mbe : 4;
        c->flush_mode = fm; c->M = M;
        c->LEAN_h = lh; c->LEAN_e = le;
        return CSEM_OK;
    }
    if (lh || le) {
        auto ok = [&](int l, int kz, int mb) {
            return l == 0 || ((l == 1 || l == 2) && (kz == 1 || kz == 2 || kz == 4) &&
                              (mb == 6 || mb == 8 || (mb == 4 && l == 2)));
        };
        if (!c->d_psiL || !ok(lh, kzh, mbh) || !ok(le, kze, mbe))
            return fail(CSEM_ERR_INVALID_ARG, "lean kernels: FP32, nx a multiple of 4, 1 or 2 cells, 1/2/4 planes, 6 or 8 (2 cells: 4, 6 or 8) blocks/SM");
    }
    if (th || te) {
        const int maxty = c->precision == 32 ? csem::tma_max_rows(c->pitch) : 0;
        auto ok = [&](int ty, int kz) { return ty == 0 || ((ty == 1 || ty == 2 || ty == 4) && ty <= maxty &&
                                                          (kz == 2 || kz == 4 || kz == 8 || kz == 16)); };
        if (!ok(th, kzh) || !ok(te, kze)) return fail(CSEM_ERR_INVALID_ARG, "staged kernels: FP32, rows 1/2/4 that fit, 2-16 planes");
    }
    if (((kzh == 16 && !th) || (kze == 16 && !te)))
        return fail(CSEM_ERR_INVALID_ARG, "16 planes per block only for the staged kernels");
    if ((vh || ve) && (c->precision != 32 || (vh && mbh == 8) || (ve && mbe == 8) || vh < 0 || vh > 1 || ve < 0 || ve > 1))
        return fail(CSEM_ERR_INVALID_ARG, "four-cell kernels: FP32 only, 4 or 6 blocks per SM");
    auto kz_ok = [](int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16; };
    auto mb_ok = [](int v) { return v == 4 || v == 6 || v == 8; };
    if (!kz_ok(kzh) || !kz_ok(kze) || !mb_ok(mbh) || !mb_ok(mbe) || !(fkz == 0 || fkz == 4 || fkz == 8 || fkz == 16) ||
        fm < 0 || fm > 3 || ((fm & 1) && c->precision != 32) || !(M == 16 || M == 32 || M == 64 || M == 128) ||
        ((fm & 2) ? 2 * M : M) + 1 > c->nslot)
        return fail(CSEM_ERR_INVALID_ARG, "launch configuration not supported by this context");
    CK(cudaDeviceSynchronize());
    c->KZ_h = kzh; c->MB_h = mbh; c->KZ_e = kze; c->MB_e = mbe;
    c->fused_kz = fkz; c->flush_mode = fm; c->M = M;
    c->FZ_by = fz_by; c->FZ_mb = fz ? fz_mb : 4; c->FZ_kz = fz ? fz_kz : 16; c->FZ_ws = ws;
    c->WAVE_lag = wv_lag; c->WAVE_kz = wv ? wv_kz : 4; c->WAVE_mb = wv ? wv_mb : 8;
    c->VEC_h = vh; c->VEC_e = ve;
    c->TMA_h = th; c->TMA_e = te;
    c->LEAN_h = lh; c->LEAN_e = le;
    return CSEM_OK;
}

int csem_autotune(csem_ctx *c, int n_src, int *kz_out, void *stream) {
    if (!c || n_src < 1 || n_src > c->max_src) return fail(CSEM_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(c->precision == 32 ? autotune_impl<float>(c, n_src, st) : autotune_impl<double>(c, n_src, st));
    if (kz_out) {
        kz_out[0] = (c->KZ_h * 16 + c->MB_h) + 256 * c->VEC_h + 1024 * c->TMA_h + 8192 * c->LEAN_h;
        kz_out[1] = (c->KZ_e * 16 + c->MB_e) + 256 * c->VEC_e + 1024 * c->TMA_e + 8192 * c->LEAN_e;
        kz_out[2] = c->M * 4 + c->flush_mode;
        kz_out[3] = (c->FZ_by || c->WAVE_lag) ? 10000 + fz_code(c) : c->fused_kz;
    }
    return CSEM_OK;
}

int csem_time_step_kernels(csem_ctx *c, int n_src, void *vol_dev, int launches, double *ms_out, void *stream) {
    if (!c || !vol_dev || !ms_out || launches < 1 || n_src < 1 || n_src > c->max_src || c->nt < 2)
        return fail(CSEM_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    return c->precision == 32 ? time_impl<float>(c, n_src, vol_dev, launches, ms_out, st)
                              : time_impl<double>(c, n_src, vol_dev, launches, ms_out, st);
}

int csem_misfit(int n, const double *d_obs, const double *d_syn, const double *w, double *resid, double *phi,
                void *stream) {
    if (n < 0 || (n > 0 && (!d_obs || !d_syn || !resid)) || !phi) return fail(CSEM_ERR_INVALID_ARG, "bad argument");
    CK(csem::launch_misfit(n, d_obs, d_syn, w, resid, phi, (cudaStream_t)stream));
    return CSEM_OK;
}

int csem_estimate_adjoint_basis(double dt, int nt, const double *freqs, int nf, double f0, double gamma,
                                int gamma_is_relative, int max_iter, double tol, double *basis_dev,
                                double *fit_residual_host, int *iters_host, void *stream) {
    if (!(dt > 0.0) || nt < 1 || !freqs || nf < 1 || nf > csem::kMaxFreq || !(f0 > 0.0) || !(gamma >= 0.0) ||
        max_iter < 0 || !basis_dev)
        return fail(CSEM_ERR_INVALID_ARG, "bad argument");
    double a[csem::kMaxFreq];
    for (int f = 0; f < nf; ++f) {
        if (!(freqs[f] > 0.0)) return fail(CSEM_ERR_INVALID_ARG, "bad frequency");
        a[f] = std::sqrt(2.0 * M_PI * freqs[f] * 2.0 * M_PI * f0);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int m = 2 * nf;
    double *scratch = nullptr;
    const size_t sbytes = (size_t)m * 2 * nt * sizeof(double) + (size_t)(m * m + 2 + m) * sizeof(double) +
                          (size_t)m * sizeof(int) + 64;
    CK(cudaMallocAsync((void **)&scratch, sbytes, st));
    double *gram = scratch + (size_t)m * 2 * nt;
    double *scal = gram + m * m;           // [0] gamma, [1..m] fit per column
    int *iters = (int *)(scal + 1 + m);
    cudaError_t e = csem::launch_basis(dt, nt, a, nf, gamma, gamma_is_relative, max_iter, tol, basis_dev, scratch,
                                       gram, scal, iters, st);
    std::vector<double> hs(1 + m);
    std::vector<int> hi(m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), scal, (1 + m) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hi.data(), iters, m * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CSEM_ERR_CUDA, std::string("adjoint basis: ") + cudaGetErrorString(e));
    if (fit_residual_host) *fit_residual_host = *std::max_element(hs.begin() + 1, hs.end());
    if (iters_host) *iters_host = *std::max_element(hi.begin(), hi.end());
    return CSEM_OK;
}

}  // extern "C"
