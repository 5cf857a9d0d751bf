// Launchers of the time-domain adjoint gradient (appendix of the paper: the
// exact adjoint of the discrete leap-frog scheme, run in reversed fictitious
// time, and the gradient as the time correlation of the two fields).
//
// Notation: E^n is the forward E after n steps (E^0 = 0), Et^m the adjoint E
// after m steps of the reversed-time run; the adjoint is driven at the
// receivers by q^{nt-1-m}, q^n = Re sum_k a_k w_{k,n}, a_k = conj(r_k) alpha_k,
// alpha_k = k_k / What_k the forward normalisation and w_{k,n} the transform
// weights.  The edge gradient is
//     dphi/dsigma_e = -1 / (2 w0 dt) sum_{m=0}^{nt-1} dV_e Et_e^m (E_e^{nt-m} - E_e^{nt-1-m}).
#pragma once
#include "csem_internal.cuh"

namespace csem {

// *step = n
cudaError_t launch_set_step(int *step, int n, cudaStream_t st);

// Adjoint series table T[m][j] = Re w_{j, nt-1-m} (j < nf), Im w_{j-nf, nt-1-m} (j >= nf),
// from w64 [nt][nf]; T is [nt][2 nf].
cudaError_t launch_td_series(const double2 *w64, double *T, int nt, int nf, cudaStream_t st);

// Emitter coefficients coef[(s*n_rec + r)*2nf + j] = Re a (j < nf), -Im a (j >= nf),
// a = conj(resid[s][r][f]) * alpha[f], so that sum_j coef T[m][j] = q^{nt-1-m}.
cudaError_t launch_td_coef(const double *resid, const double2 *alpha, double *coef, int S, int n_rec, int nf,
                           cudaStream_t st);

// acc[e] += sum_s sum_{t<cnt} Et^{m0+t}_e (E^{nt-m0-t}_e - E^{nt-m0-t-1}_e), e over the 3 vol entries.
//  F: forward ring, E^n of source s at F + s*f_stride + (n % f_slots)*n3;
//  A: adjoint ring, Et^m at A + s*a_stride + (m % a_slots)*n3;  n3 = 3 vol (a multiple of 4).
// Within one call the products are summed in R with compensation, then added to acc in double.
template <typename R>
cudaError_t launch_td_corr(const R *F, long long f_stride, int f_slots, const R *A, long long a_stride, int a_slots,
                           int S, long long n3, int nt, int m0, int cnt, double *acc, cudaStream_t st);

// pe[e] = (R)(scale * acc[e]) over n elements
template <typename R>
cudaError_t launch_td_edges(const double *acc, double scale, long long n, R *pe, cudaStream_t st);

// Cell gradient from per-edge values pe [3][vol] (the edge form divided by dV_e),
// accumulated into grad (kern_aux.cu; the mapping of csem_gradient).
template <typename R>
cudaError_t launch_grad_cells(const GeoD &g, const R *rho, const R *pe, int wrt, bool vti, R *grad, cudaStream_t st);

}  // namespace csem
