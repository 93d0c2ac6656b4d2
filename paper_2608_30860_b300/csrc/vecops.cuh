// Host launchers of the HBM-bound vector kernels (vecops.cu) and the small eigensolver (hess.cu).
#pragma once
#include "common.cuh"

constexpr int DOT_BLOCKS = 592;   // 4 CTAs per SM on 148 SMs; partial buffers hold DOT_BLOCKS * k

// out[i] (+)= <V_i, w> for i < k (V_i = V + i * vstride); partial: DOT_BLOCKS * k scratch
int vec_dot_block(const cplx* V, long long vstride, int k, const cplx* w, long long len, cplx* out,
                  cplx* partial, int accumulate, cudaStream_t s);
// y = (keep_y ? y : 0) + sign * sum_i h[i] V_i   (k <= 128)
int vec_gemv(cplx* y, const cplx* V, long long vstride, int k, const cplx* h, long long len, double sign,
             int keep_y, cudaStream_t s);
// hcol[0..k) += h2; hcol[k] = sqrt(nrm2); inv = 1 / hcol[k] (0 on breakdown, recorded in brk[0] = k
// when brk is non-null and still 0)
int vec_finish_column(cplx* hcol, const cplx* h2, int k, const cplx* nrm2, cplx* inv, cudaStream_t s,
                      int* brk = nullptr);
int vec_scale_dev(cplx* x, long long len, const cplx* a, cudaStream_t s);
int vec_scale_copy(cplx* y, const cplx* x, long long len, cplx a, cudaStream_t s);
int vec_axpby(cplx* y, const cplx* x, long long len, cplx a, cplx b, cudaStream_t s);
int mat_trace(const cplx* X, int n, cplx* out, cudaStream_t s);
int mat_div_by_dev(cplx* out, const cplx* X, long long len, const cplx* tr, cudaStream_t s, int real_only = 0);
int mat_hermitize(cplx* Y, const cplx* X, int n, cudaStream_t s);
// out[0] = max |x_e|, out[1] = ||x||_2 ; part: 2 * DOT_BLOCKS doubles
int vec_norms(const cplx* x, long long len, double* part, double* out, cudaStream_t s);
int mat_eye(cplx* X, int n, cplx a, cudaStream_t s);
// R <- R + R^dag (in place)
int mat_add_adjoint(cplx* R, int n, cudaStream_t s);
// gauge split in place: L_k += c_k I, then H += (1/2i) sum_k (c_k^* L_k - c_k L_k^dag) (c_dev: d complex)
int gauge_split(cplx* H, cplx* L, int n, int d, const cplx* c_dev, cudaStream_t s);
int mat_add_diag_dev(cplx* X, int n, const cplx* a, double scale, cudaStream_t s);
int mat_transpose(cplx* Y, const cplx* X, int n, cudaStream_t s);
// T = upper(A); out[1] = ||strictly-lower(A)||_F
int mat_take_upper(cplx* T, const cplx* A, int n, double* part, double* out, cudaStream_t s);
int mat_min_abs_re_diag(const cplx* T, int n, double* out, cudaStream_t s);
// X_ij /= (T_ii + conj(T_jj) - 2 shift)
int mat_eig_divide(cplx* X, const cplx* T, int n, double shift, cudaStream_t s);

// small dense eigensolver for an m x m upper-Hessenberg matrix (m <= 64), hess.cu
int hess_eig(const cplx* H, int ldh, int m, cplx* evals, cplx* evecs, int* info, cudaStream_t s);

// triangular Lyapunov (T - s I) X + X (T - s I)^dag = C, in place, sylvester.cu
int trisylv_f64(const cplx* T, cplx* X, int n, cplx s, cudaStream_t st);

// general small Schur/eigen kernel (hess.cu): A column-major (lda); hess_in = 1 if A is
// already upper Hessenberg; order: 0 none, 1 largest |.| first, 2 nearest 1 first (the nsel
// leading positions); outputs ordered evals, evecs (vector p contiguous), T and Z
// (column-major, ld m; nullable).
int small_schur(const cplx* A, int lda, int m, int hess_in, int order, int nsel, cplx* evals, cplx* evecs,
                cplx* Tout, cplx* Zout, int* info, cudaStream_t s);

