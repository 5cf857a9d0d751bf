// Adjoint-source basis without any device allocation.
//
// csem_estimate_adjoint_basis obtains its CGNR work vectors with
// cudaMallocAsync.  This variant takes them from one file-scope device array
// instead, so that a caller who must not allocate device memory can still
// build the basis: for example an application whose device memory is owned by
// another allocator (a framework's caching pool or a fixed arena that must not
// be bypassed), or code on a path where an allocation's implicit
// synchronisation or failure is not acceptable.  The array is sized for
// nt <= kNoAllocMaxNt and n_freq <= kMaxFreq and stays resident on every device
// that loads the library until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/csem.h"
#include "csem_internal.cuh"

namespace {

constexpr int kNoAllocMaxNt = 32768;
constexpr int kNoAllocMaxCols = 2 * csem::kMaxFreq;
// layout: [cols][2][nt] CG vectors | [cols][cols] Gram matrix | [1 + cols] scalars | [cols] int iteration counts
constexpr size_t kVecDoubles = (size_t)kNoAllocMaxCols * 2 * kNoAllocMaxNt;
constexpr size_t kGramDoubles = (size_t)kNoAllocMaxCols * kNoAllocMaxCols;
constexpr size_t kScalDoubles = 1 + kNoAllocMaxCols;
constexpr size_t kIterDoubles = (kNoAllocMaxCols + 1) / 2;   // ints packed two per double
constexpr size_t kScratchDoubles = kVecDoubles + kGramDoubles + kScalDoubles + kIterDoubles;

__device__ __align__(256) double g_basis_scratch[kScratchDoubles];   // 8 MiB + a few KiB

// Host code cannot use g_basis_scratch's name as a device address.  Resolve it
// on every call, with the caller's device current: once the module is loaded this
// is a table lookup, and a fresh lookup stays right after cudaDeviceReset (which
// unloads the module; the next call loads it again at a new address).
int scratch_for_current_device(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_basis_scratch);
    if (e != cudaSuccess || !p) {
        return csem::set_last_error(CSEM_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    }
    *out = (double *)p;
    return CSEM_OK;
}

}  // namespace

extern "C" int csem_estimate_adjoint_basis_noalloc(double dt, int nt, const double *freqs, int nf, double f0,
                                                   double gamma, int gamma_is_relative, int max_iter, double tol,
                                                   double *basis_dev, double *fit_residual_host, int *iters_host,
                                                   void *stream) {
    if (!(dt > 0.0) || nt < 1 || !freqs || nf < 1 || !(f0 > 0.0) || !(gamma >= 0.0) || max_iter < 0 || !basis_dev) {
        return csem::set_last_error(CSEM_ERR_INVALID_ARG, "bad argument");
    }
    if (nt > kNoAllocMaxNt || nf > csem::kMaxFreq) {
        return csem::set_last_error(CSEM_ERR_INVALID_ARG, "csem_estimate_adjoint_basis_noalloc supports nt <= " + std::to_string(kNoAllocMaxNt) +
                        " and n_freq <= " + std::to_string(csem::kMaxFreq) + " (got nt = " + std::to_string(nt) +
                        ", n_freq = " + std::to_string(nf) + ")");
    }
    double a[csem::kMaxFreq];
    for (int f = 0; f < nf; ++f) {
        if (!(freqs[f] > 0.0)) {
            return csem::set_last_error(CSEM_ERR_INVALID_ARG, "bad frequency");
        }
        a[f] = std::sqrt(2.0 * M_PI * freqs[f] * 2.0 * M_PI * f0);
    }
    double *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc != CSEM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int m = 2 * nf;
    double *vec = base;
    double *gram = base + kVecDoubles;
    double *scal = gram + kGramDoubles;
    int *iters = (int *)(scal + kScalDoubles);
    // The basis kernels write every value of the array they later read, so a clear is
    // not needed for the result; it is kept, limited to the part this call uses (its
    // m CG vector pairs and the Gram/scalar/count block), so that a kernel fault can
    // never show a previous call's numbers.
    cudaError_t e = cudaMemsetAsync(vec, 0, (size_t)m * 2 * nt * sizeof(double), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(gram, 0, (kGramDoubles + kScalDoubles + kIterDoubles) * sizeof(double), st);
    if (e == cudaSuccess)
        e = csem::launch_basis(dt, nt, a, nf, gamma, gamma_is_relative, max_iter, tol, basis_dev, vec, gram, scal,
                               iters, st);
    double hs[1 + kNoAllocMaxCols];
    int hi[kNoAllocMaxCols];
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, scal, (1 + m) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hi, iters, m * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        return csem::set_last_error(CSEM_ERR_CUDA, std::string("adjoint basis (no-alloc): ") + cudaGetErrorString(e));
    }
    double fit = 0.0;
    int its = 0;
    for (int j = 0; j < m; ++j) {
        fit = hs[1 + j] > fit ? hs[1 + j] : fit;
        its = hi[j] > its ? hi[j] : its;
    }
    if (fit_residual_host) *fit_residual_host = fit;
    if (iters_host) *iters_host = its;
    return CSEM_OK;
}
