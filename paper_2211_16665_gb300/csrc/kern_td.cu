// Kernels of the time-domain adjoint gradient (appendix): the adjoint series
// and emitter coefficients, the time correlation of forward and adjoint E,
// and the per-edge result.  The stepping itself reuses the forward kernels.
#include "csem_internal.cuh"
#include "csem_td.cuh"

namespace csem {

namespace {

__global__ void k_set_step(int *step, int n) { *step = n; }

__global__ void k_td_series(const double2 *w64, double *T, int nt, int nf) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nt * 2 * nf) return;
    const int j = (int)(t % (2 * nf));
    const int m = (int)(t / (2 * nf));
    const double2 w = w64[(long long)(nt - 1 - m) * nf + (j % nf)];
    T[t] = (j < nf) ? w.x : w.y;
}

__global__ void k_td_coef(const double *resid, const double2 *alpha, double *coef, int n, int nf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;   // (s, r, f)
    if (t >= n) return;
    const int f = t % nf, sr = t / nf;
    const double rr = resid[2 * t], ri = -resid[2 * t + 1];   // conj(r)
    const double2 al = alpha[f];
    coef[(long long)sr * 2 * nf + f] = rr * al.x - ri * al.y;          // Re a
    coef[(long long)sr * 2 * nf + nf + f] = -(rr * al.y + ri * al.x);  // -Im a
}

template <typename R> struct Lanes;
template <> struct Lanes<float> { typedef float4 V; static constexpr int W = 4; };
template <> struct Lanes<double> { typedef double2 V; static constexpr int W = 2; };

template <typename R> __device__ __forceinline__ R lane(const typename Lanes<R>::V &v, int l);
template <> __device__ __forceinline__ float lane<float>(const float4 &v, int l) {
    return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w;
}
template <> __device__ __forceinline__ double lane<double>(const double2 &v, int l) { return l == 0 ? v.x : v.y; }

// One thread per W consecutive entries of the 3 vol block; the forward snapshots are
// walked downwards in n and the adjoint ones upwards in m, each loaded once.
template <typename R>
__global__ void __launch_bounds__(256) k_td_corr(const R *F, long long fs, int fsl, const R *A, long long as, int asl,
                                                 int S, long long nv, int nt, int m0, int cnt, double *acc) {
    typedef typename Lanes<R>::V V;
    constexpr int W = Lanes<R>::W;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nv) return;
    double tot[W];
#pragma unroll
    for (int l = 0; l < W; ++l) tot[l] = 0.0;
    for (int s = 0; s < S; ++s) {
        const V *Fs = reinterpret_cast<const V *>(F + (long long)s * fs);
        const V *As = reinterpret_cast<const V *>(A + (long long)s * as);
        int fslot = (nt - m0) % fsl, aslot = m0 % asl;
        V hi = __ldg(Fs + (long long)fslot * nv + e);
        R sum[W], cmp[W];
#pragma unroll
        for (int l = 0; l < W; ++l) { sum[l] = R(0); cmp[l] = R(0); }
#pragma unroll 4
        for (int t = 0; t < cnt; ++t) {
            fslot = (fslot == 0 ? fsl : fslot) - 1;
            const V lo = __ldg(Fs + (long long)fslot * nv + e);
            const V a = __ldg(As + (long long)aslot * nv + e);
            aslot = (aslot + 1 == asl) ? 0 : aslot + 1;
#pragma unroll
            for (int l = 0; l < W; ++l) {   // compensated sum of a (hi - lo)
                const R y = lane<R>(a, l) * (lane<R>(hi, l) - lane<R>(lo, l)) - cmp[l];
                const R u = sum[l] + y;
                cmp[l] = (u - sum[l]) - y;
                sum[l] = u;
            }
            hi = lo;
        }
#pragma unroll
        for (int l = 0; l < W; ++l) tot[l] += (double)sum[l] - (double)cmp[l];
    }
#pragma unroll
    for (int l = 0; l < W; ++l) acc[e * W + l] += tot[l];
}

template <typename R>
__global__ void k_td_edges(const double *acc, double scale, long long n, R *pe) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) pe[t] = (R)(scale * acc[t]);
}

}  // namespace

cudaError_t launch_set_step(int *step, int n, cudaStream_t st) {
    k_set_step<<<1, 1, 0, st>>>(step, n);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_td_series(const double2 *w64, double *T, int nt, int nf, cudaStream_t st) {
    const long long n = (long long)nt * 2 * nf;
    k_td_series<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w64, T, nt, nf);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_td_coef(const double *resid, const double2 *alpha, double *coef, int S, int n_rec, int nf,
                           cudaStream_t st) {
    const int n = S * n_rec * nf;
    if (n == 0) return cudaSuccess;
    k_td_coef<<<(n + 255) / 256, 256, 0, st>>>(resid, alpha, coef, n, nf);
    g_launches++;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_td_corr(const R *F, long long f_stride, int f_slots, const R *A, long long a_stride, int a_slots,
                           int S, long long n3, int nt, int m0, int cnt, double *acc, cudaStream_t st) {
    constexpr int W = Lanes<R>::W;
    if (cnt <= 0) return cudaSuccess;
    if (n3 % 4 != 0 || m0 < 0 || m0 + cnt > nt || cnt + 1 > f_slots || cnt + 1 > a_slots) return cudaErrorInvalidValue;
    const long long nv = n3 / W;
    k_td_corr<R><<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(F, f_stride, f_slots, A, a_stride, a_slots, S, nv, nt,
                                                                m0, cnt, acc);
    g_launches++;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_td_edges(const double *acc, double scale, long long n, R *pe, cudaStream_t st) {
    k_td_edges<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(acc, scale, n, pe);
    g_launches++;
    return cudaGetLastError();
}

template cudaError_t launch_td_corr<float>(const float *, long long, int, const float *, long long, int, int,
                                           long long, int, int, int, double *, cudaStream_t);
template cudaError_t launch_td_corr<double>(const double *, long long, int, const double *, long long, int, int,
                                            long long, int, int, int, double *, cudaStream_t);
template cudaError_t launch_td_edges<float>(const double *, double, long long, float *, cudaStream_t);
template cudaError_t launch_td_edges<double>(const double *, double, long long, double *, cudaStream_t);

}  // namespace csem
