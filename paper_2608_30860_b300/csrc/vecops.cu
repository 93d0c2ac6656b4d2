// HBM-bound vector kernels of the Krylov loops: Hilbert-Schmidt inner products against a
// block of basis vectors (classical Gram-Schmidt, applied twice), the matching update
// w -= V h, Ritz-vector formation, traces, hermitisation and norms.  Every reduction is a
// fixed-order two-stage tree (per-CTA partials, then one CTA), so results are reproducible.
#include "common.cuh"
#include "vecops.cuh"

namespace {

constexpr int RT = 256;        // threads per CTA
constexpr int KB = 8;          // basis vectors per pass of the dot kernel

__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// partial[blk * k + i] = sum over this CTA's slice of conj(V_i[e]) * w[e]
__global__ void __launch_bounds__(RT) k_block_dot(const cplx* __restrict__ V, long long vstride, int k,
                                                  const cplx* __restrict__ w, long long len,
                                                  cplx* __restrict__ partial) {
    __shared__ cplx red[RT / 32][KB];
    const int i0 = blockIdx.y * KB;
    const int kk = min(KB, k - i0);
    cplx acc[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = cmake(0.0, 0.0);
    for (long long e = (long long)blockIdx.x * RT + threadIdx.x; e < len; e += (long long)gridDim.x * RT) {
        cplx x = w[e];
#pragma unroll
        for (int i = 0; i < KB; ++i) {
            if (i < kk) {
                cplx v = V[(long long)(i0 + i) * vstride + e];
                acc[i].x += v.x * x.x + v.y * x.y;
                acc[i].y += v.x * x.y - v.y * x.x;
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        cplx s = warp_sum(acc[i]);
        if (lane == 0) red[wid][i] = s;
    }
    __syncthreads();
    if (threadIdx.x < kk) {
        cplx s = cmake(0.0, 0.0);
        for (int q = 0; q < RT / 32; ++q) s = cadd(s, red[q][threadIdx.x]);
        partial[(long long)blockIdx.x * k + i0 + threadIdx.x] = s;
    }
}

// out[i] (+)= sum_b partial[b * k + i]
__global__ void k_reduce_partials(const cplx* __restrict__ partial, int nblk, int k, cplx* __restrict__ out,
                                  int accumulate) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        cplx s = cmake(0.0, 0.0);
        for (int b = 0; b < nblk; ++b) s = cadd(s, partial[(long long)b * k + i]);
        out[i] = accumulate ? cadd(out[i], s) : s;
    }
}

// y[e] = beta*y[e] + sign * sum_i h[i] V_i[e]
__global__ void __launch_bounds__(RT) k_gemv(cplx* __restrict__ y, const cplx* __restrict__ V, long long vstride,
                                             int k, const cplx* __restrict__ h, long long len, double sign,
                                             int keep_y) {
    __shared__ cplx hs[128];
    for (int i = threadIdx.x; i < k; i += RT) hs[i] = h[i];
    __syncthreads();
    for (long long e = (long long)blockIdx.x * RT + threadIdx.x; e < len; e += (long long)gridDim.x * RT) {
        cplx s = cmake(0.0, 0.0);
        for (int i = 0; i < k; ++i) cfma(s, hs[i], V[(long long)i * vstride + e]);
        cplx out = cscale(s, sign);
        if (keep_y) out = cadd(y[e], out);
        y[e] = out;
    }
}

// Arnoldi column finalisation: hcol[i] += h2[i]; beta = ||w|| (from |w|^2 in nrm2);
// hcol[k] = beta; inv[0] = 1/beta.
// Completes Hessenberg column k-1 (k entries from the two Gram-Schmidt passes, then the norm) and
// the scale 1/h_{k,k-1} of the next basis vector.  With brk non-null, breakdown is detected here:
// h_{k,k-1} <= 1e-13 max(1, max_i |h_{i,k-1}|) records k in brk[0] (if still 0) and sets the scale
// to 0, so that the remaining steps of the cycle carry zero vectors and the host reads the step
// count once per cycle instead of once per step.
__global__ void k_finish_column(cplx* hcol, const cplx* h2, int k, const cplx* nrm2, cplx* inv, int* brk) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) hcol[i] = cadd(hcol[i], h2[i]);
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = sqrt(fmax(nrm2[0].x, 0.0));
        double hmax = 0.0;
        for (int i = 0; i < k; ++i) hmax = fmax(hmax, hypot(hcol[i].x, hcol[i].y));
        bool dead = !(b > 0.0);
        if (brk) {
            dead = dead || brk[0] != 0 || !(b > 1e-13 * fmax(1.0, hmax));
            if (dead && brk[0] == 0) brk[0] = k;
        }
        hcol[k] = cmake(b, 0.0);
        inv[0] = cmake(dead ? 0.0 : 1.0 / b, 0.0);
    }
}

// x[e] *= s[0]  (device scalar)
__global__ void k_scale_dev(cplx* x, long long len, const cplx* s) {
    cplx a = s[0];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
        x[e] = cmul(a, x[e]);
}

__global__ void k_scale_copy(cplx* y, const cplx* x, long long len, cplx a) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
        y[e] = cmul(a, x[e]);
}

// y = a*x + b*y
__global__ void k_axpby(cplx* y, const cplx* x, long long len, cplx a, cplx b) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
        y[e] = cadd(cmul(a, x[e]), cmul(b, y[e]));
}

// single-CTA trace: out[0] = sum_i X[i][i]
__global__ void k_trace(const cplx* X, int n, cplx* out) {
    __shared__ cplx red[32];
    cplx s = cmake(0.0, 0.0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = cadd(s, X[(long long)i * n + i]);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        cplx t = cmake(0.0, 0.0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = cadd(t, red[q]);
        out[0] = t;
    }
}

// out = X / tr[0]  (tr a device scalar; phase fix of a Ritz vector); real_only divides by Re tr[0]
__global__ void k_div_by_dev(cplx* out, const cplx* X, long long len, const cplx* tr, int real_only) {
    cplx t = tr[0];
    if (real_only) t.y = 0.0;
    double d = cabs2(t);
    cplx inv = d > 0.0 ? cmake(t.x / d, -t.y / d) : cmake(0.0, 0.0);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
        out[e] = cmul(inv, X[e]);
}

// Y = (X + X^dag)/2 (out of place; Y != X)
__global__ void k_hermitize(cplx* __restrict__ Y, const cplx* __restrict__ X, int n) {
    long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / n), j = (int)(e % n);
        cplx a = X[e], b = X[(long long)j * n + i];
        Y[e] = cmake(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
}

// per-CTA partial max |x| and sum |x|^2  -> part[2*blk], part[2*blk+1]
__global__ void __launch_bounds__(RT) k_norms_partial(const cplx* x, long long len, double* part) {
    __shared__ double rm[RT / 32], rs[RT / 32];
    double m = 0.0, s = 0.0;
    for (long long e = (long long)blockIdx.x * RT + threadIdx.x; e < len; e += (long long)gridDim.x * RT) {
        double a2 = cabs2(x[e]);
        m = fmax(m, a2);
        s += a2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) { rm[threadIdx.x >> 5] = m; rs[threadIdx.x >> 5] = s; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = 0.0, S = 0.0;
        for (int q = 0; q < RT / 32; ++q) { M = fmax(M, rm[q]); S += rs[q]; }
        part[2 * blockIdx.x] = M;
        part[2 * blockIdx.x + 1] = S;
    }
}

__global__ void k_norms_final(const double* part, int nblk, double* out) {
    if (threadIdx.x == 0) {
        double M = 0.0, S = 0.0;
        for (int b = 0; b < nblk; ++b) { M = fmax(M, part[2 * b]); S += part[2 * b + 1]; }
        out[0] = sqrt(M);
        out[1] = sqrt(S);
    }
}

// X = a * I
__global__ void k_eye(cplx* X, int n, cplx a) {
    long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / n), j = (int)(e % n);
        X[e] = (i == j) ? a : cmake(0.0, 0.0);
    }
}

// X[i][i] += a[0] * s   (device scalar a)
__global__ void k_add_diag_dev(cplx* X, int n, const cplx* a, double s) {
    cplx v = cscale(a[0], s);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        X[(long long)i * n + i] = cadd(X[(long long)i * n + i], v);
}

// Y = X^T (out of place)
__global__ void k_transpose(cplx* __restrict__ Y, const cplx* __restrict__ X, int n) {
    __shared__ cplx tile[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int i = by + r, j = bx + threadIdx.x;
        if (i < n && j < n) tile[r][threadIdx.x] = X[(long long)i * n + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int i = bx + r, j = by + threadIdx.x;
        if (i < n && j < n) Y[(long long)i * n + j] = tile[threadIdx.x][r];
    }
}

// T := upper triangle of A (strictly-lower part zeroed); part gets per-CTA sum |lower|^2
__global__ void __launch_bounds__(RT) k_take_upper(cplx* __restrict__ T, const cplx* __restrict__ A, int n,
                                                   double* part) {
    __shared__ double rs[RT / 32];
    long long len = (long long)n * n;
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * RT + threadIdx.x; e < len; e += (long long)gridDim.x * RT) {
        int i = (int)(e / n), j = (int)(e % n);
        cplx a = A[e];
        if (i > j) { s += cabs2(a); a = cmake(0.0, 0.0); }
        T[e] = a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) rs[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0;
        for (int q = 0; q < RT / 32; ++q) S += rs[q];
        part[2 * blockIdx.x] = 0.0;
        part[2 * blockIdx.x + 1] = S;
    }
}

// min_i |Re T_ii|
__global__ void k_min_abs_re_diag(const cplx* T, int n, double* out) {
    __shared__ double red[32];
    double m = 1e300;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, fabs(T[(long long)i * n + i].x));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = 1e300;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) M = fmin(M, red[q]);
        out[0] = M;
    }
}

// X_ij /= (T_ii + conj(T_jj) - 2 shift)  (eigenbasis divide; T's diagonal holds the eigenvalues)
__global__ void k_eig_divide(cplx* X, const cplx* T, int n, double shift) {
    const long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const cplx si = T[(long long)i * n + i], sj = T[(long long)j * n + j];
        X[e] = cdiv(X[e], cmake(si.x + sj.x - 2.0 * shift, si.y - sj.y));
    }
}

inline int grid_for(long long len) {
    long long g = (len + RT - 1) / RT;
    if (g > 148 * 8) g = 148 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int vec_dot_block(const cplx* V, long long vstride, int k, const cplx* w, long long len, cplx* out,
                  cplx* partial, int accumulate, cudaStream_t s) {
    const int nblk = DOT_BLOCKS;
    dim3 grid(nblk, (k + KB - 1) / KB);
    k_block_dot<<<grid, RT, 0, s>>>(V, vstride, k, w, len, partial); lb_note_launch();
    k_reduce_partials<<<1, 128, 0, s>>>(partial, nblk, k, out, accumulate); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int vec_gemv(cplx* y, const cplx* V, long long vstride, int k, const cplx* h, long long len, double sign,
             int keep_y, cudaStream_t s) {
    k_gemv<<<grid_for(len), RT, 0, s>>>(y, V, vstride, k, h, len, sign, keep_y); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int vec_finish_column(cplx* hcol, const cplx* h2, int k, const cplx* nrm2, cplx* inv, cudaStream_t s, int* brk) {
    k_finish_column<<<1, 128, 0, s>>>(hcol, h2, k, nrm2, inv, brk); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int vec_scale_dev(cplx* x, long long len, const cplx* a, cudaStream_t s) {
    k_scale_dev<<<grid_for(len), RT, 0, s>>>(x, len, a); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int vec_scale_copy(cplx* y, const cplx* x, long long len, cplx a, cudaStream_t s) {
    k_scale_copy<<<grid_for(len), RT, 0, s>>>(y, x, len, a); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int vec_axpby(cplx* y, const cplx* x, long long len, cplx a, cplx b, cudaStream_t s) {
    k_axpby<<<grid_for(len), RT, 0, s>>>(y, x, len, a, b); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_trace(const cplx* X, int n, cplx* out, cudaStream_t s) {
    k_trace<<<1, 256, 0, s>>>(X, n, out); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_div_by_dev(cplx* out, const cplx* X, long long len, const cplx* tr, cudaStream_t s, int real_only) {
    k_div_by_dev<<<grid_for(len), RT, 0, s>>>(out, X, len, tr, real_only); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_hermitize(cplx* Y, const cplx* X, int n, cudaStream_t s) {
    k_hermitize<<<grid_for((long long)n * n), RT, 0, s>>>(Y, X, n); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int vec_norms(const cplx* x, long long len, double* part, double* out, cudaStream_t s) {
    k_norms_partial<<<DOT_BLOCKS, RT, 0, s>>>(x, len, part); lb_note_launch();
    k_norms_final<<<1, 32, 0, s>>>(part, DOT_BLOCKS, out); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Gauge of the no-jump / jump split (Remark "Non-uniqueness of the decomposition"):
// (1) L~_k = L_k + c_k I in place; (2) H~ = H + (1/2i) sum_k (conj(c_k) L~_k - c_k L~_k^dag) in place.
__global__ void k_gauge_jumps(cplx* L, int n, int d, const cplx* c) {
    const long long nn = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)d * n; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), i = (int)(e % n);
        cplx* p = L + k * nn + (long long)i * n + i;
        *p = cadd(*p, c[k]);
    }
}
__global__ void k_gauge_hamiltonian(cplx* H, const cplx* Lt, int n, int d, const cplx* c) {
    const long long nn = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        cplx acc = cmake(0, 0);
        for (int k = 0; k < d; ++k) {
            const cplx a = Lt[k * nn + e];                           // L~_k[i][j]
            const cplx bdag = cconj(Lt[k * nn + (long long)j * n + i]);   // (L~_k^dag)[i][j]
            acc = cadd(acc, csub(cmul(cconj(c[k]), a), cmul(c[k], bdag)));
        }
        // (1/2i) acc = -i acc / 2
        H[e] = cadd(H[e], cmake(0.5 * acc.y, -0.5 * acc.x));
    }
}

int gauge_split(cplx* H, cplx* L, int n, int d, const cplx* c_dev, cudaStream_t s) {
    k_gauge_jumps<<<grid_for((long long)d * n), RT, 0, s>>>(L, n, d, c_dev); lb_note_launch();
    k_gauge_hamiltonian<<<grid_for((long long)n * n), RT, 0, s>>>(H, L, n, d, c_dev); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// R <- R + R^dag in place: one thread per pair i <= j (the pair is read before either is written)
__global__ void k_add_adjoint(cplx* R, int n) {
    const long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (i > j) continue;
        const cplx a = R[e], b = R[(long long)j * n + i];
        const cplx v = cadd(a, cconj(b));
        R[e] = v;
        if (i != j) R[(long long)j * n + i] = cconj(v);
        else R[e] = cmake(v.x, 0.0);
    }
}

int mat_add_adjoint(cplx* R, int n, cudaStream_t s) {
    k_add_adjoint<<<grid_for((long long)n * n), RT, 0, s>>>(R, n); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_eye(cplx* X, int n, cplx a, cudaStream_t s) {
    k_eye<<<grid_for((long long)n * n), RT, 0, s>>>(X, n, a); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_add_diag_dev(cplx* X, int n, const cplx* a, double scale, cudaStream_t s) {
    k_add_diag_dev<<<(n + 255) / 256, 256, 0, s>>>(X, n, a, scale); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_transpose(cplx* Y, const cplx* X, int n, cudaStream_t s) {
    dim3 g((n + 31) / 32, (n + 31) / 32);
    k_transpose<<<g, dim3(32, 8), 0, s>>>(Y, X, n); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_take_upper(cplx* T, const cplx* A, int n, double* part, double* out, cudaStream_t s) {
    k_take_upper<<<DOT_BLOCKS, RT, 0, s>>>(T, A, n, part); lb_note_launch();
    k_norms_final<<<1, 32, 0, s>>>(part, DOT_BLOCKS, out); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_eig_divide(cplx* X, const cplx* T, int n, double shift, cudaStream_t s) {
    k_eig_divide<<<grid_for((long long)n * n), RT, 0, s>>>(X, T, n, shift); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mat_min_abs_re_diag(const cplx* T, int n, double* out, cudaStream_t s) {
    k_min_abs_re_diag<<<1, 256, 0, s>>>(T, n, out); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
