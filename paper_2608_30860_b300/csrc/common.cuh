// Shared device/host helpers for the Lindblad library (complex128 as double2: x = re, y = im).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

typedef double2 cplx;

#define LB_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) {                                                       \
            fprintf(stderr, "lindblad: CUDA error %s at %s:%d\n", cudaGetErrorString(_e), \
                    __FILE__, __LINE__);                                               \
            return LB_CUDA_ERROR;                                                      \
        }                                                                              \
    } while (0)

__host__ __device__ __forceinline__ cplx cmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// c += a * b
__host__ __device__ __forceinline__ void cfma(cplx& c, cplx a, cplx b) {
    c.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
    c.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
}
// a / b with scaling (Smith's algorithm)
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    } else {
        double r = b.x / b.y, den = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
    }
}

// GEMM operand modes: element op(A)[i][k] of a row-major matrix with leading dimension ld
enum { OP_N = 0, OP_T = 1, OP_C = 2 };

struct ZGemmArgs {
    int M, N, K;
    const cplx* A; long long lda, strideA; int opA;
    const cplx* B; long long ldb, strideB; int opB;
    cplx* C; long long ldc, strideC;
    cplx alpha, beta;
    int batch;    // number of (A_b, B_b) pairs
    int reduce;   // 1: C = alpha * sum_b op(A_b) op(B_b) + beta C ; 0: C_b = alpha op(A_b) op(B_b) + beta C_b
    int herm;     // 1 (reduce = 1, M = N): the result is Hermitian (alpha, beta real, C Hermitian on entry):
                  // only the tiles on and above the diagonal are computed, the rest is mirrored; 2: the same
                  // and the diagonal's imaginary part is set to zero (an exactly Hermitian result)
};

// C[i][j] = conj(C[j][i]) for i > j, and Im C[i][i] = 0 when real_diag (n x n, leading dimension ld)
int mat_mirror_lower(cplx* C, int n, long long ld, cudaStream_t s, int real_diag = 0);

// host launchers (defined in the .cu files)
int zgemm_f64(const ZGemmArgs& a, cudaStream_t s);

// counts every kernel launch issued by the library (lb_launch_count in the C ABI)
void lb_note_launch();

// raises a kernel's dynamic shared-memory limit on the current device, once per (kernel, device);
// thread-safe; returns 0 on success
int lb_smem_attr(const void* kernel, int bytes);
