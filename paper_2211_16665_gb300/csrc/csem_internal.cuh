// Internal declarations shared by the CUDA translation units of the engine.
// Layout of one source's state in HBM (all per-source blocks are contiguous):
//   H       [3][vol]         Hx, Hy, Hz on the padded node lattice,
//                            index (k*NY + j)*pitch + i, NY = ny+1, NZ = nz+1
//   ering   [nslot][3][vol]  E snapshots: E^n (Ex, Ey, Ez) in slot n mod nslot,
//                            nslot = M + 1 for a transform block of M steps
//   H2      [3][vol]         second H buffer (the fused step reads one, writes the other)
//   psi     CPML memory arrays, each only inside the slab of its axis, six per axis:
//           x-slabs [NZ][NY][2 npml]   : psi(Hy,dEz/dx) psi(Hz,dEy/dx) psi(Ey,dHz/dx) psi(Ez,dHy/dx) + H pair B
//           y-slabs [NZ][2 npml][pitch]: psi(Hx,dEz/dy) psi(Hz,dEx/dy) psi(Ex,dHz/dy) psi(Ez,dHx/dy) + H pair B
//           z-slabs [2 npml][NY][pitch]: psi(Hx,dEy/dz) psi(Hy,dEx/dz) psi(Ex,dHy/dz) psi(Ey,dHx/dz) + H pair B
//           (arrays [0],[1] and [4],[5] are the two buffers of the H-update memory)
//   acc     [3][nf][vol] complex damped-transform accumulators (the caller's volume buffer)
//   comp    [3][nf][vol] complex Kahan compensation (context workspace, FP32 only)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

namespace csem {

extern std::atomic<long long> g_launches;   // kernels launched by this library

template <typename R> __device__ __forceinline__ R ldg_r(const R *p) { return __ldg(p); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Bounded wait on an mbarrier phase, shared by the bulk-copy kernels: true once the phase of
// this parity has completed; false after about kWaitNs of the global timer (or 2^26 polls),
// so a kernel whose copies never arrive reports a timeout instead of hanging.
constexpr unsigned long long kWaitNs = 1000000000ull;
__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_done(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = gtimer_ns();
    for (int it = 0; it < (1 << 26); ++it) {
        if (mbar_done(bar, parity)) return true;
        if ((it & 255) == 255 && gtimer_ns() - t0 > kWaitNs) return false;
    }
    return false;
}
// Status bits the kernels raise in the context's device word (read and cleared by csem_check).
constexpr int kErrNonfinite = 1;     // a resistivity was non-positive or non-finite
constexpr int kErrFlushWait = 2;     // a bulk-copy transform flush gave up waiting for its copies
constexpr int kErrStagedWait = 4;    // a row-staged H / E step kernel gave up waiting
constexpr int kErrOnepassWait = 8;   // the fused one-pass step kernel gave up waiting
constexpr int kErrWaveWait = 16;     // an E tile of the wave-ordered step gave up waiting for H
constexpr int kMaxWaveChunks = 4096; // z blocks the wave-ordered step's counters cover

template <typename R> struct C2;
template <> struct C2<float> { typedef float2 T; };
template <> struct C2<double> { typedef double2 T; };

constexpr int kMaxFreq = 8;
constexpr int kBlock = 256;
constexpr int kMaxBlockSteps = 128;  // largest transform block (snapshots per flush)

// Slab index of a half node i (between nodes i and i+1) on an axis of n cells:
// the first npml and the last npml half nodes lie in the CPML.
__host__ __device__ inline int slab_half(int i, int n, int npml) {
    if (i < npml) return i;
    if (i >= n - npml && i < n) return i - n + 2 * npml;
    return -1;
}
// Slab index of an interior node i: nodes 1..npml-1 and n-npml+1..n-1 lie in the CPML
// (node 0 / n carry no update, the interface nodes npml and n-npml have zero damping).
__host__ __device__ inline int slab_node(int i, int n, int npml) {
    if (i >= 1 && i < npml) return i;
    if (i > n - npml && i < n) return i - n + 2 * npml - 1;
    return -1;
}

template <typename R>
struct AxisTab {          // per-axis stepping tables (device, type R)
    const R *ih_h, *ih_n; // 1/h at half nodes [n], 1/h~ at nodes [n+1]
    const R *b_h, *a_h;   // CPML recursion at half nodes [n]
    const R *b_n, *a_n;   // CPML recursion at nodes [n+1]
};

struct GeoTab {            // per-axis FP32 widths for the fused one-pass step (padded to 16-byte groups)
    const float *h;       // primal width at half nodes [n]
    const float *s;       // sum of the two primal widths next to a node [n+1] (2 x the dual width)
};

template <typename R>
struct StepParams {
    int nx, ny, nz, NX, NY, NZ, pitch, npml;
    long long plane, vol;          // pitch*NY, plane*NZ
    AxisTab<R> ax, ay, az;
    R *H;                          // [S][3][vol]
    R *H2;                         // [S][3][vol] second H buffer (fused step)
    int fused_kz;                  // > 0: one fused H+E kernel per step with this z blocking
    R *ering;                      // [S][nslot][3][vol]
    long long ering_stride;        // nslot*3*vol
    int nslot;                     // transform block M + 1
    R *psi;                        // [S][psi_stride]
    long long psi_stride, sx, sy, sz;
    const R *cE;                   // [3][vol] dt/eps on each E edge
    R cH;                          // dt/mu0
    const int *step;               // device step counter (chunk base)
    int KZ_h, KZ_e;                // z planes per thread of the H / E kernels (1, 2, 4 or 8)
    int MB_h, MB_e;                // minimum resident blocks per SM the kernels are compiled for (4, 6, 8)
    int VEC_h, VEC_e;              // 1: FP32 kernels with four cells per thread along x
    int TMA_h, TMA_e;              // > 0: FP32 bulk-copy-staged kernels over this many rows per block
    int LEAN_h, LEAN_e;            // > 0: lean FP32 kernels with this many cells per thread (1 or 2)
    AxisTab<R> lx, ly, lz;         // the stepping tables padded to 16-byte groups (lean kernels)
    const R *lzero;                // 4 zeros, 16-byte aligned (lean kernels)
    R *psiL;                       // [S][12][vol] CPML memory in the field layout (lean kernels)
    const R *cEm;                  // [3][vol] dt/eps, zero on the PEC edges (lean kernels)
    // fused one-pass FP32 step (kern_fz.cu): FZ_by rows per block (0: off), FZ_mb resident
    // blocks per SM, FZ_kz planes per z block; q = V sigma per cell on the lattice (qv = qh
    // unless the medium is VTI), per-axis widths, 2 w0 dt
    int FZ_by, FZ_mb, FZ_kz;
    int FZ_ws;                     // 1: the warp-specialised fused kernel with the same shape fields
    // wave-ordered step (kern_lean.cu): the lean H and E tiles in one launch, E lagging H by
    // WAVE_lag z blocks of WAVE_kz planes (WAVE_lag 0: off); wave: [2 + kMaxWaveChunks] counters
    int WAVE_kz, WAVE_mb, WAVE_lag;
    unsigned *wave;
    const float *qh, *qv;
    GeoTab gx, gy, gz;
    float k2w0dt;
    int *err;                      // device status word (kErr* bits)
    int fault_tx;                  // test hook: extra bytes the first barrier arm of each block of a
                                   // bulk-copy kernel expects, so that its bounded wait runs out
    int nf;
    const typename C2<R>::T *w;    // [nt][nf] exp((-1+i) a_k n dt)
    typename C2<R>::T *acc;        // [S][3][nf][vol] or nullptr
    typename C2<R>::T *comp;       // Kahan compensation or nullptr
    // source injection into E^{n+1}, applied by the E kernel: taps sorted by
    // lattice column; colmap[s*colmap_stride + (j*pitch + i)] = (first tap, count)
    const int2 *colmap;            // nullptr: no injection
    long long colmap_stride;       // plane, or 0 when every source shares the taps
    // tflag[s*tflag_stride + j*nseg + i/32] != 0: the 32 columns from i (rounded down) of row j
    // hold a tap (lean kernels read the column map only there)
    const unsigned char *tflag;
    long long tflag_stride;        // ny*nseg, or 0 when every source shares the taps
    int nseg;                      // ceil(nx / 32)
    // lean E kernel: the increment -dt/eps J'^{n+1/2} of tap u of source s at step jstep of the
    // current graph chunk, inc[(jstep*S + s)*inc_ntl + u] (FP32, rounded once from FP64), and
    // tapk[s*itap_stride + u] = (plane k of the tap) * 4 + component
    float *inc;
    const int *tapk;
    int inc_ntl;
    const struct Tap *itaps;
    int itap_stride, n_emit, J;
    const double *coef;            // [S][n_emit][J]
    const double *T;               // [nt][J]
};

struct Tap {                       // one trilinear tap of a point operator (32 bytes)
    long long idx;                 // lattice index inside a component block
    double w;                      // weight (divided by the edge's dual volume for injection)
    int comp;                      // 0,1,2
    int emit;                      // emitter (series) id for injection, receiver id for sampling
    int pad0, pad1;
};

template <typename R>
struct PointParams {
    const R *cE;
    const int *step;
    int nt, nf;
    // sampling (receivers shared by all sources), done in the transform flush
    int n_rec; const Tap *rtaps;   // [n_rec][8]
    double2 *racc;                 // [S][n_rec][nf]
    const double2 *w64;            // [nt][nf]
    double *trace;                 // [S][n_rec][nt] or nullptr
    // injection into E^{n+1}
    int n_itaps; const Tap *itaps; // source s uses itaps[s*itap_stride .. + n_itaps)
    int itap_stride;
    int n_emit, J;
    const double *coef;            // [S][n_emit][J]
    const double *T;               // [nt][J]
};

// ---- launchers (kern_step.cu) ----
// which: bit 0 = H half-step, bit 2 = E step (with the source injection)
template <typename R>
cudaError_t launch_step(const StepParams<R> &p, const PointParams<R> &q, int S, int jstep, cudaStream_t st,
                        int which = 5);
// transform (and receiver sampling) of snapshots n0 .. n0+cnt-1, n0 = *step + n0_off
template <typename R>
cudaError_t launch_dft(const StepParams<R> &p, const PointParams<R> &q, int S, int n0_off, int cnt, bool vol,
                       bool kahan, cudaStream_t st);
cudaError_t launch_advance(int *step, int by, cudaStream_t st);
// FP32 flush of exactly cnt (16 or 32) snapshots through bulk copies into shared memory;
// a bounded barrier wait that gives up raises bit 1 of *err
cudaError_t launch_dft_bulk(const StepParams<float> &p, const PointParams<float> &q, int S, int n0_off, int cnt,
                            bool kahan, int *err, cudaStream_t st);
cudaError_t prepare_bulk_flush();
// fused H+E step (kern_fused.cu), kz in {4, 8, 16}
template <typename R>
cudaError_t launch_fused(const StepParams<R> &p, int S, int jstep, int kz, cudaStream_t st);
cudaError_t prepare_fused_all();
// fused one-pass FP32 step (kern_fz.cu): nx even, (by, mb) in {(4,4), (4,6), (8,2), (8,3)}, kz planes per z block
cudaError_t launch_step_fz(const StepParams<float> &p, int S, int jstep, cudaStream_t st);
bool fz_supported(int by, int mb, int kz);
// warp-specialised fused FP32 step (kern_fz.cu, FZ_ws = 1): nx even, (by, mb) in {(4,2), (4,3), (6,2),
// (8,1), (8,2)}, kz planes per z block; reads the masked dt/eps and the slab CPML memory
cudaError_t launch_step_ws(const StepParams<float> &p, int S, int jstep, cudaStream_t st);
bool ws_supported(int by, int mb, int kz);
// FP32 H / E kernels with four cells per thread (kern_vec.cu), kz in {1,2,4,8}, mb in {4,6}
// lean FP32 H / E kernels (kern_lean.cu), nx % 4 == 0, w (cells per thread) in {1,2}, kz in {1,2,4},
// mb (resident 128-thread blocks per SM) in {6,8} for w = 1 and {4,6,8} for w = 2
cudaError_t launch_field_lean(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h, int w, int kz,
                              int mb);
// wave-ordered FP32 step (kern_lean.cu): the lean H and E tiles (2 cells per thread) of one step in one
// launch, WAVE_kz in {2, 4}, WAVE_mb in {6, 8}, WAVE_lag >= 1; an E tile that gives up waiting raises
// kErrWaveWait
cudaError_t launch_step_wave(const StepParams<float> &p, int S, int jstep, cudaStream_t st);
bool wave_supported(const StepParams<float> &p, int kz, int mb);
// cEm = cE with the PEC edges zeroed
cudaError_t launch_mask_coef(const StepParams<float> &p, const float *cE, float *cEm, cudaStream_t st);
// p.inc for the steps jstep in [0, nsteps) after *p.step (zero past nt)
cudaError_t launch_tap_inc(const StepParams<float> &p, int S, int nsteps, int nt, cudaStream_t st);
cudaError_t launch_field_vec(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h, int kz, int mb);
// FP32 bulk-copy-staged H / E kernels (kern_tma.cu): ty rows per block in {1,2,4}, kz planes per chunk
cudaError_t launch_field_tma(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h, int kz, int ty,
                             int *err);
cudaError_t prepare_tma();
int tma_max_rows(int pitch);
size_t fused_smem_bytes(int real_size);

// ---- launchers (kern_aux.cu) ----
struct GeoD {                      // double-precision geometry for set-up and gradient kernels
    int nx, ny, nz, NX, NY, NZ, pitch;
    long long plane, vol;
    const double *hx, *hy, *hz;    // primal widths [n]
};
// q = V sigma per cell on the lattice (sigma_h into qh; sigma_v into qv when qv is not NULL)
cudaError_t launch_qcell(const GeoD &g, const float *rho, const float *rho_z, float *qh, float *qv, cudaStream_t st);
template <typename R>
// dt/eps on every edge from the cell resistivity (rho_z on the z edges: rho_v of a VTI medium, else rho)
cudaError_t launch_coef_init(const GeoD &g, const R *rho, const R *rho_z, R *cE, double two_w0_dt, int *bad_flag,
                             cudaStream_t st);
template <typename R>
cudaError_t launch_finalize_volume(typename C2<R>::T *acc, const typename C2<R>::T *comp, long long vol, int S,
                                   int nf, const double2 *alpha, cudaStream_t st);
cudaError_t launch_finalize_receivers(const double2 *racc, double *out, int S, int n_rec, int nf,
                                      const double2 *alpha, cudaStream_t st);
cudaError_t launch_adjoint_coef(const double *resid, double *coef, int S, int n_rec, int nf,
                                const double2 *kf, double inv_dt, cudaStream_t st);
template <typename R>
cudaError_t launch_gradient(const GeoD &g, const R *rho, const typename C2<R>::T *E, const typename C2<R>::T *V,
                            int S, int nf, int wrt, bool vti, R *edge_scratch, R *grad, cudaStream_t st);
cudaError_t launch_scatter_int2(int2 *dst, const long long *pos, const int2 *val, int n, cudaStream_t st);
cudaError_t launch_misfit(int n, const double *d_obs, const double *d_syn, const double *w, double *resid,
                          double *phi, cudaStream_t st);
cudaError_t launch_basis(double dt, int nt, const double *a, int nf, double gamma, int gamma_rel, int max_iter,
                         double tol, double *basis, double *scratch, double *gram, double *out_scalars,
                         int *out_iters, cudaStream_t st);

// records msg as the calling thread's csem_last_error() text and returns code
int set_last_error(int code, const std::string &msg);

}  // namespace csem
