// Small dense eigenproblems of the Krylov loops (m <= 64, FP64, one warp, shared memory):
// Ritz values and vectors of an Arnoldi cycle (Alg. 4) and the ordered Schur form needed by
// the Krylov-Schur thick restart of Alg. 5.
//
//   1. (general input) Householder reduction to upper-Hessenberg form, Z accumulated;
//   2. complex Schur form by the implicitly shifted single-shift QR algorithm (Wilkinson
//      shift from the trailing 2 x 2, exceptional shifts after 10 and 20 stalled sweeps,
//      deflation on negligible subdiagonals);
//   3. optional reordering of the Schur form by adjacent swaps: each swap is the Givens
//      rotation that maps the 2 x 2 block's second eigenvector onto e1;
//   4. eigenvectors of the triangular factor by back substitution, mapped back with Z and
//      normalised to unit 2-norm.
// Rotations are applied with the 32 lanes splitting the row / column index.  The QR sweep
// count is capped at 30 m; info = 1 reports a stall.
#include "common.cuh"
#include "vecops.cuh"

#include "small_schur.cuh"

namespace {

__global__ void k_small_schur(const cplx* __restrict__ Ain, int lda, int m, int hess_in, int order, int nsel,
                              cplx* __restrict__ evals, cplx* __restrict__ evecs, cplx* __restrict__ Tout,
                              cplx* __restrict__ Zout, int* info) {
    extern __shared__ __align__(16) unsigned char hsm[];
    cplx* A = reinterpret_cast<cplx*>(hsm);   // m x m row-major, row stride m + 1
    cplx* Z = A + m * (m + 1);                  // m x m row-major, row stride m + 1
    cplx* Vt = Z + m * (m + 1);                 // eigenvectors of T, row p = vector p, stride m + 1
    __shared__ cplx hv[64];
    __shared__ cplx rot_s;
    __shared__ double rot_c;
    small_schur_warp(Ain, lda, m, hess_in, order, nsel, evals, evecs, Tout, Zout, info, A, Z, Vt, hv, rot_s, rot_c);
}

}  // namespace

int small_schur(const cplx* A, int lda, int m, int hess_in, int order, int nsel, cplx* evals, cplx* evecs,
                cplx* Tout, cplx* Zout, int* info, cudaStream_t s) {
    if (m < 1 || m > 64) return -1;
    size_t smem = 3 * (size_t)m * (m + 1) * sizeof(cplx);
    if (lb_smem_attr((const void*)k_small_schur, 3 * 64 * 65 * (int)sizeof(cplx))) return -1;
    k_small_schur<<<1, 32, smem, s>>>(A, lda, m, hess_in, order, nsel, evals, evecs, Tout, Zout, info); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int hess_eig(const cplx* H, int ldh, int m, cplx* evals, cplx* evecs, int* info, cudaStream_t s) {
    return small_schur(H, ldh, m, 1, 0, 0, evals, evecs, nullptr, nullptr, info, s);
}
