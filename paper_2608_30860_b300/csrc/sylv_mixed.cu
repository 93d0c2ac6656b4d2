// Mixed-precision triangular Lyapunov solve (T - sI) X + X (T - sI)^dag = C in Schur
// coordinates (the Bartels-Stewart back substitution of App. A.1.1), for the tensor-core path.
//
// Blocks of 128 x 128 are swept by anti-diagonals from the bottom-right corner.  Per
// anti-diagonal w two launches:
//   (1) the left-looking update of every block (I, J) on w,
//         C_IJ -= sum_{K>I} T_IK X_KJ + sum_{L>J} X_IL T_JL^dag,
//       one tcgen05 CTA per block (tc_gemm.cu, wavefront mode, BF16 hi/lo operands -- BF16 keeps
//       FP32's exponent range, so the unknown magnitude of X needs no scale);
//   (2) the leaf solve of each block in FP32 on the CUDA cores: a left-looking sweep over the
//       block's 255 anti-diagonals (4 threads per entry).  The leaf writes X_IJ back (complex128)
//       and refreshes the BF16 planes of X and X^T that the later updates read.
#include <cuda_bf16.h>

#include "lb_internal.cuh"
#include "tc_gemm.cuh"
#include "vecops.cuh"

struct SylvMixed {
    int np = 0, nb = 0;
    __nv_bfloat16* Tp = nullptr;    // 4 x np x np, rows of T (unshifted)
    __nv_bfloat16* Xp = nullptr;    // 4 x np x np, rows of X
    __nv_bfloat16* XTp = nullptr;   // 4 x np x np, rows of X^T
    float2* Tf = nullptr;           // np x np, T in FP32 (row-major)
    float2* Ttf = nullptr;          // np x np, T^T in FP32
    tc::Maps maps{};                // 0: T, 1: X^T, 2: X
};

namespace {

constexpr int LB = 128;   // wavefront block
constexpr int LEAF_THREADS = 512;   // 4 threads per entry of an anti-diagonal (<= 128 entries)
// shared-memory row pitch in complex floats.  A warp holds 8 anti-diagonal entries (slot s,
// a = a0 + s, b = S - a) x 4 threads t; its loads X[a+1+t][b] and X[a][b+1+t] sit at word offsets
// (pitch-1) s + pitch t and (pitch-1) s + t.  With pitch = 5 (mod 32) both sets cover the 32
// eight-byte bank pairs exactly once.
constexpr int PITCH = LB + 5;

struct f2 {
    float x, y;
};
__device__ __forceinline__ f2 fmk(float a, float b) { return f2{a, b}; }

__device__ __forceinline__ f2 f2ld(const float2* p) { const float2 v = __ldg(p); return fmk(v.x, v.y); }

// Leaf of one 128 x 128 block (I, J) of the wavefront: A X + X B^dag = C with A = T_II - sI,
// B = T_JJ - sI (upper triangular), C already updated by the tensor-core step.  Left-looking
// anti-diagonal sweep over the whole block: the entries (a, b) with a + b = S are independent and
//   X_ab = (C_ab - sum_{r>a} A_ar X_rb - sum_{r>b} X_ar conj(B_br)) / (A_aa + conj(B_bb)),
// each dot product of the same length 254 - S, split over 4 threads and reduced by shuffles.
// A is kept in shared memory as a packed upper triangle; B rows are read through L1/L2.
__global__ void __launch_bounds__(LEAF_THREADS, 1)
k_sylv_leaf128(const float2* __restrict__ Tf, const float2* __restrict__ Ttf, int ldf, cplx* __restrict__ X, int n,
               float sh, int wave, int nb, __nv_bfloat16* __restrict__ Xp, __nv_bfloat16* __restrict__ XTp,
               int np) {
    extern __shared__ __align__(16) unsigned char smraw[];
    f2(*Xs)[PITCH] = reinterpret_cast<f2(*)[PITCH]>(smraw);                       // 128 x PITCH
    f2* Ap = reinterpret_cast<f2*>(smraw + sizeof(f2) * LB * PITCH);              // packed upper triangle
    const int t = blockIdx.x + max(0, wave - (nb - 1));
    const int I = nb - 1 - t, J = nb - 1 - (wave - t);
    const int r0 = I * LB, c0 = J * LB;
    const int br = min(LB, n - r0), bc = min(LB, n - c0);
    const int tid = threadIdx.x;
    (void)Ttf;

    for (int e = tid; e < LB * LB; e += LEAF_THREADS) {
        const int p = e / LB, q = e % LB;
        cplx v = (p < br && q < bc) ? X[(long long)(r0 + p) * n + c0 + q] : cmake(0, 0);
        Xs[p][q] = fmk((float)v.x, (float)v.y);
        if (q >= p) {
            f2 a = (p < br && q < br) ? f2ld(Tf + (long long)(r0 + p) * ldf + r0 + q) : fmk(0.f, 0.f);
            if (q == p) a.x -= sh;
            Ap[p * LB - (p * (p - 1)) / 2 + (q - p)] = a;
        }
    }
    __syncthreads();

    const int slot = tid >> 2, t4 = tid & 3;
    for (int S = (br - 1) + (bc - 1); S >= 0; --S) {
        const int a = max(0, S - (bc - 1)) + slot;
        const int b = S - a;
        const bool valid = a < br && b >= 0 && a <= S;
        f2 acc = fmk(0.f, 0.f);
        if (valid) {
            // four independent partial sums so that four loads are in flight
            f2 p[4] = {fmk(0.f, 0.f), fmk(0.f, 0.f), fmk(0.f, 0.f), fmk(0.f, 0.f)};
            const int arow = a * LB - (a * (a - 1)) / 2 - a;      // Ap index of A[a][r] = arow + r
            int r = a + 1 + t4;
            for (; r + 12 < br; r += 16) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const f2 m = Ap[arow + r + 4 * u], x = Xs[r + 4 * u][b];
                    p[u].x += m.x * x.x - m.y * x.y;
                    p[u].y += m.x * x.y + m.y * x.x;
                }
            }
            for (; r < br; r += 4) {
                const f2 m = Ap[arow + r], x = Xs[r][b];
                p[0].x += m.x * x.x - m.y * x.y;
                p[0].y += m.x * x.y + m.y * x.x;
            }
            const float2* brow = Tf + (long long)(c0 + b) * ldf + c0;
            r = b + 1 + t4;
            for (; r + 12 < bc; r += 16) {
                f2 m[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) m[u] = f2ld(brow + r + 4 * u);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const f2 x = Xs[a][r + 4 * u];
                    p[u].x += x.x * m[u].x + x.y * m[u].y;
                    p[u].y += x.y * m[u].x - x.x * m[u].y;
                }
            }
            for (; r < bc; r += 4) {
                const f2 x = Xs[a][r], m = f2ld(brow + r);
                p[1].x += x.x * m.x + x.y * m.y;
                p[1].y += x.y * m.x - x.x * m.y;
            }
            acc = fmk((p[0].x + p[1].x) + (p[2].x + p[3].x), (p[0].y + p[1].y) + (p[2].y + p[3].y));
        }
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
        if (valid && t4 == 0) {
            const f2 da = Ap[a * LB - (a * (a - 1)) / 2];
            f2 db = f2ld(Tf + (long long)(c0 + b) * ldf + c0 + b);
            db.x -= sh;
            const float dr = da.x + db.x, di = da.y - db.y;   // A_aa + conj(B_bb)
            const float inv = 1.0f / (dr * dr + di * di);
            const f2 v = fmk(Xs[a][b].x - acc.x, Xs[a][b].y - acc.y);
            Xs[a][b] = fmk((v.x * dr + v.y * di) * inv, (v.y * dr - v.x * di) * inv);
        }
        __syncthreads();
    }
    // write back: complex128 block and the BF16 hi/lo planes of X (rows), lanes along q ...
    const long long ps = (long long)np * np;
    for (int e = tid; e < LB * LB; e += LEAF_THREADS) {
        const int p = e / LB, q = e % LB;
        if (p >= br || q >= bc) continue;
        const f2 v = Xs[p][q];
        X[(long long)(r0 + p) * n + c0 + q] = cmake((double)v.x, (double)v.y);
        const __nv_bfloat16 rh = __float2bfloat16(v.x), ih = __float2bfloat16(v.y);
        const __nv_bfloat16 rl = __float2bfloat16(v.x - __bfloat162float(rh));
        const __nv_bfloat16 il = __float2bfloat16(v.y - __bfloat162float(ih));
        const long long o = (long long)(r0 + p) * np + c0 + q;
        Xp[o] = rh; Xp[ps + o] = rl; Xp[2 * ps + o] = ih; Xp[3 * ps + o] = il;
    }
    // ... and of X^T (rows = columns of X), lanes along p so that the stores stay contiguous
    for (int e = tid; e < LB * LB; e += LEAF_THREADS) {
        const int q = e / LB, p = e % LB;
        if (p >= br || q >= bc) continue;
        const f2 v = Xs[p][q];
        const __nv_bfloat16 rh = __float2bfloat16(v.x), ih = __float2bfloat16(v.y);
        const __nv_bfloat16 rl = __float2bfloat16(v.x - __bfloat162float(rh));
        const __nv_bfloat16 il = __float2bfloat16(v.y - __bfloat162float(ih));
        const long long ot = (long long)(c0 + q) * np + r0 + p;
        XTp[ot] = rh; XTp[ps + ot] = rl; XTp[2 * ps + ot] = ih; XTp[3 * ps + ot] = il;
    }
}

// FP32 copies of T (row-major and transposed, zero padding), read by the leaf kernel through L1
__global__ void k_t_to_f32(const cplx* __restrict__ T, int n, float2* __restrict__ Tf, float2* __restrict__ Ttf,
                           int ld) {
    const long long len = (long long)ld * ld;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ld), j = (int)(e % ld);
        const cplx v = (i < n && j < n) ? T[(long long)i * n + j] : cmake(0, 0);
        Tf[e] = make_float2((float)v.x, (float)v.y);
        Ttf[(long long)j * ld + i] = make_float2((float)v.x, (float)v.y);
    }
}

constexpr size_t LEAF_SMEM = sizeof(f2) * LB * PITCH + sizeof(f2) * (LB * (LB + 1) / 2);

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

size_t sylv_mixed_bytes(int n) {
    const size_t np = (size_t)round_up(n, LB);
    return 3 * (4 * np * np * sizeof(__nv_bfloat16) + 256) + 2 * (np * np * sizeof(float2) + 256);
}

int sylv_mixed_prepare(lb_handle_s* h, char* base, cudaStream_t s) {
    SylvMixed* m = new SylvMixed();
    h->sylv = m;
    m->np = round_up(h->n, LB);
    m->nb = m->np / LB;
    const size_t np = m->np;
    const size_t plane_bytes = 4 * np * np * sizeof(__nv_bfloat16);
    auto carve = [&](size_t bytes) {
        char* p = base;
        base += (bytes + 255) & ~size_t(255);
        return p;
    };
    m->Tp = reinterpret_cast<__nv_bfloat16*>(carve(plane_bytes));
    m->Xp = reinterpret_cast<__nv_bfloat16*>(carve(plane_bytes));
    m->XTp = reinterpret_cast<__nv_bfloat16*>(carve(plane_bytes));
    m->Tf = reinterpret_cast<float2*>(carve(np * np * sizeof(float2)));
    m->Ttf = reinterpret_cast<float2*>(carve(np * np * sizeof(float2)));
    k_t_to_f32<<<1184, 256, 0, s>>>(h->T, h->n, m->Tf, m->Ttf, (int)np);
    lb_note_launch();
    if (cudaMemsetAsync(m->Xp, 0, plane_bytes, s) != cudaSuccess) return -1;
    if (cudaMemsetAsync(m->XTp, 0, plane_bytes, s) != cudaSuccess) return -1;
    if (tc_split_planes_bf16(h->T, h->n, h->n, h->n, 0, m->Tp, (int)np, (long long)np * np, s)) return -1;
    if (tc_make_map(&m->maps.m[0], m->Tp, (int)np, (int)np, 1, (int)np, 1)) return -1;
    if (tc_make_map(&m->maps.m[1], m->XTp, (int)np, (int)np, 1, (int)np, 1)) return -1;
    if (tc_make_map(&m->maps.m[2], m->Xp, (int)np, (int)np, 1, (int)np, 1)) return -1;
    m->maps.m[3] = m->maps.m[0];
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_sylv_leaf128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LEAF_SMEM) !=
            cudaSuccess)
            return -1;
        attr = true;
    }
    h->mixed_sylv_ready = true;
    return 0;
}

// Solves (T - shift I) X + X (T - shift I)^dag = C in place (X holds C on entry).
int trisylv_mixed(lb_handle_s* h, cudaStream_t s, cplx* X, double shift) {
    SylvMixed* m = h->sylv;
    if (!m) return -1;
    const int nb = m->nb;
    tc::Params p{};
    p.M = h->n;
    p.N = h->n;
    p.nseg = 2;
    p.seg[0] = tc::Seg{0, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0, tc::SIGN_NORMAL};   // T_IK (X^T)_JK
    p.seg[1] = tc::Seg{2, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, tc::SIGN_CONJ_B};   // X_IL conj(T_JL)
    p.npairs = 3;
    p.out = X;
    p.ldo = h->n;
    p.alpha = -1.0;
    p.scale = nullptr;
    p.accumulate = 1;
    p.err = h->dinfo + 8;
    p.fmt = 1;
    p.nb = nb;
    for (int w = 0; w <= 2 * nb - 2; ++w) {
        const int lo = w - (nb - 1) > 0 ? w - (nb - 1) : 0;
        const int hi = w < nb - 1 ? w : nb - 1;
        const int cnt = hi - lo + 1;
        if (w > 0) {
            p.wave = w;
            if (tc_gemm_launch(m->maps, p, cnt, 1, s)) return -1;
        }
        k_sylv_leaf128<<<cnt, LEAF_THREADS, LEAF_SMEM, s>>>(m->Tf, m->Ttf, m->np, X, h->n, (float)shift, w, nb, m->Xp,
                                                             m->XTp, m->np);
        lb_note_launch();
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

void sylv_mixed_release(lb_handle_s* h) {
    delete h->sylv;
    h->sylv = nullptr;
}
