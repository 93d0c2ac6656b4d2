// FP64 complex GEMM on the CUDA cores (the all-FP64 path, the set-up products and the FP64
// residual L(rho) of the stopping test).
//
//   C = alpha * sum_b op(A_b) op(B_b) + beta * C      (reduce = 1: the jump-term sum over j)
//   C_b = alpha * op(A_b) op(B_b) + beta * C_b         (reduce = 0: batched)
//
// op in {N, T, C(onjugate transpose)} on row-major operands.  64 x 64 output tile per CTA,
// K step 8, 256 threads with a 4 x 4 register tile each; the operand tiles are staged in
// shared memory with the load pattern chosen per op so that global reads stay coalesced.
#include "common.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 8;

__device__ __forceinline__ cplx load_op(const cplx* __restrict__ P, long long ld, int op, int r, int c) {
    // element [r][c] of op(P)
    if (op == OP_N) return P[(long long)r * ld + c];
    cplx v = P[(long long)c * ld + r];
    if (op == OP_C) v.y = -v.y;
    return v;
}

__global__ void __launch_bounds__(256) zgemm_f64_kernel(ZGemmArgs a) {
    __shared__ cplx As[BK][BM + 1];
    __shared__ cplx Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int bz = blockIdx.z;
    if (a.herm && blockIdx.y > blockIdx.x) return;   // strictly below the diagonal: mirrored afterwards

    cplx acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cmake(0.0, 0.0);

    const int b_begin = a.reduce ? 0 : bz;
    const int b_end = a.reduce ? a.batch : bz + 1;
    for (int b = b_begin; b < b_end; ++b) {
        const cplx* A = a.A + (long long)b * a.strideA;
        const cplx* B = a.B + (long long)b * a.strideB;
        for (int k0 = 0; k0 < a.K; k0 += BK) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                int idx = tid + r * 256;
                int mm, kk;
                if (a.opA == OP_N) { mm = idx / BK; kk = idx % BK; }
                else { mm = idx % BM; kk = idx / BM; }
                int gm = m0 + mm, gk = k0 + kk;
                As[kk][mm] = (gm < a.M && gk < a.K) ? load_op(A, a.lda, a.opA, gm, gk) : cmake(0.0, 0.0);
                int nn;
                if (a.opB == OP_N) { nn = idx % BN; kk = idx / BN; }
                else { nn = idx / BK; kk = idx % BK; }
                int gn = n0 + nn;
                gk = k0 + kk;
                Bs[kk][nn] = (gn < a.N && gk < a.K) ? load_op(B, a.ldb, a.opB, gk, gn) : cmake(0.0, 0.0);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < BK; ++k) {
                cplx av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) cfma(acc[i][j], av[i], bv[j]);
            }
            __syncthreads();
        }
    }
    cplx* C = a.C + (a.reduce ? 0 : (long long)bz * a.strideC);
    const bool use_beta = (a.beta.x != 0.0 || a.beta.y != 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= a.N) continue;
            cplx v = cmul(a.alpha, acc[i][j]);
            long long off = (long long)gm * a.ldc + gn;
            if (use_beta) v = cadd(v, cmul(a.beta, C[off]));
            C[off] = v;
        }
    }
}

// C[i][j] = conj(C[j][i]) below the diagonal, 32 x 32 tiles through shared memory (coalesced both ways);
// real_diag: also Im C[i][i] = 0, so that the result is exactly Hermitian.  (The Krylov solvers keep the
// computed diagonal: zeroing its rounding-level imaginary part inside the Phi-Arnoldi operator stalled the
// FP64 steady state of slowly mixing Kerr cats at ~1e-6.)
__global__ void k_mirror_lower(cplx* C, int n, long long ld, int real_diag) {
    __shared__ cplx t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;   // destination tile (bi, bj), bi >= bj
    if (bi < bj) return;
    const int tx = threadIdx.x;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int r = bj * 32 + yy, c = bi * 32 + tx;   // source: the tile (bj, bi) above the diagonal
        if (r < n && c < n) t[yy][tx] = C[(long long)r * ld + c];
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int r = bi * 32 + yy, c = bj * 32 + tx;
        if (r < n && c < n && r > c) C[(long long)r * ld + c] = cconj(t[tx][yy]);
        if (real_diag && r < n && r == c) C[(long long)r * ld + c].y = 0.0;   // a Hermitian diagonal is real
    }
}

}  // namespace

int mat_mirror_lower(cplx* C, int n, long long ld, cudaStream_t s, int real_diag) {
    const int nt = (n + 31) / 32;
    k_mirror_lower<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(C, n, ld, real_diag); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int zgemm_f64(const ZGemmArgs& a, cudaStream_t s) {
    if (a.M <= 0 || a.N <= 0) return 0;
    if (a.herm && (a.M != a.N || !a.reduce)) return -1;
    dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, a.reduce ? 1 : a.batch);
    zgemm_f64_kernel<<<grid, 256, 0, s>>>(a); lb_note_launch();
    if (cudaGetLastError() != cudaSuccess) return -1;
    return a.herm ? mat_mirror_lower(a.C, a.M, a.ldc, s, a.herm == 2) : 0;
}
