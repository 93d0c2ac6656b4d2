// lindbladian_apply_noalloc: R = L(X) from H and the jumps directly, with no handle, no caller
// workspace and no allocation.  Its two n x n complex128 scratch matrices (G and one jump
// product) live in a file-scope device array of fixed size, so sizes above
// LB_NOALLOC_NMAX are refused.  Every scratch element is written before it is read: nothing
// has to start at zero.  Calls on one device share the array, so calls that overlap in time
// (two streams, two host threads) race; the caller serialises them.
#include <mutex>

#include "common.cuh"
#include "lindblad.h"

namespace {

constexpr int kNmax = LB_NOALLOC_NMAX;
constexpr int kMaxDevices = 64;

// 2 * 512^2 complex128 = 8 MiB of module memory, reserved when the module loads
static __device__ __align__(256) cplx g_noalloc_scratch[2 * (size_t)kNmax * kNmax];

cplx* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

__global__ void k_minus_i(const cplx* __restrict__ H, cplx* __restrict__ G, long long nn) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x)
        G[e] = cmake(H[e].y, -H[e].x);
}

// device address of the scratch array on the current device, looked up once per device
cplx* scratch_address() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        g_scratch_addr[dev] = static_cast<cplx*>(p);
    }
    return g_scratch_addr[dev];
}

int gemm1(cudaStream_t s, cplx* C, const cplx* A, int opA, const cplx* B, int opB, int n, cplx alpha, cplx beta) {
    ZGemmArgs g{};
    g.M = g.N = g.K = n;
    g.A = A; g.lda = n; g.strideA = 0; g.opA = opA;
    g.B = B; g.ldb = n; g.strideB = 0; g.opB = opB;
    g.C = C; g.ldc = n; g.strideC = 0;
    g.alpha = alpha; g.beta = beta;
    g.batch = 1;
    g.reduce = 0;
    return zgemm_f64(g, s);
}

}  // namespace

extern "C" lb_status lindbladian_apply_noalloc(const void* H_dev, const void* L_dev, int n, int d, const void* X_dev,
                                               void* R_dev, void* stream) {
    if (!H_dev || !L_dev || !X_dev || !R_dev || n < 2 || d < 1) return LB_INVALID_ARG;
    if (n > kNmax) return LB_WORKSPACE_TOO_SMALL;
    cplx* G = scratch_address();
    if (!G) return LB_CUDA_ERROR;
    cplx* P = G + (size_t)n * n;
    cudaStream_t s = (cudaStream_t)stream;
    const cplx* H = static_cast<const cplx*>(H_dev);
    const cplx* L = static_cast<const cplx*>(L_dev);
    const cplx* X = static_cast<const cplx*>(X_dev);
    cplx* R = static_cast<cplx*>(R_dev);
    const long long nn = (long long)n * n;
    // G = -iH - 1/2 sum_j L_j^dag L_j  (Eq. (2)), one reduced batched GEMM over the jumps
    k_minus_i<<<(int)((nn + 255) / 256 < 1184 ? (nn + 255) / 256 : 1184), 256, 0, s>>>(H, G, nn);
    lb_note_launch();
    if (cudaGetLastError() != cudaSuccess) return LB_CUDA_ERROR;
    ZGemmArgs g{};
    g.M = g.N = g.K = n;
    g.A = L; g.lda = n; g.strideA = nn; g.opA = OP_C;
    g.B = L; g.ldb = n; g.strideB = nn; g.opB = OP_N;
    g.C = G; g.ldc = n; g.strideC = 0;
    g.alpha = cmake(-0.5, 0.0); g.beta = cmake(1.0, 0.0);
    g.batch = d;
    g.reduce = 1;
    if (zgemm_f64(g, s)) return LB_CUDA_ERROR;
    // R = G X + X G^dag + sum_j L_j X L_j^dag  (Eq. (1))
    if (gemm1(s, R, G, OP_N, X, OP_N, n, cmake(1, 0), cmake(0, 0))) return LB_CUDA_ERROR;
    if (gemm1(s, R, X, OP_N, G, OP_C, n, cmake(1, 0), cmake(1, 0))) return LB_CUDA_ERROR;
    for (int j = 0; j < d; ++j) {
        if (gemm1(s, P, L + j * nn, OP_N, X, OP_N, n, cmake(1, 0), cmake(0, 0))) return LB_CUDA_ERROR;
        if (gemm1(s, R, P, OP_N, L + j * nn, OP_C, n, cmake(1, 0), cmake(1, 0))) return LB_CUDA_ERROR;
    }
    return LB_OK;
}
