// Mixed-precision triangular Lyapunov solve (T - sI) X + X (T - sI)^dag = C in Schur
// coordinates (the Bartels-Stewart back substitution of App. A.1.1), for the tensor-core path.
//
// Blocks of 128 x 128 are swept by anti-diagonals from the bottom-right corner.  Per
// anti-diagonal w two launches:
//   (1) the left-looking update of every block (I, J) on w,
//         C_IJ -= sum_{K>I} T_IK X_KJ + sum_{L>J} X_IL T_JL^dag,
//       one tcgen05 CTA per block (tc_gemm.cu, wavefront mode, BF16 hi/lo operands -- BF16 keeps
//       FP32's exponent range, so the unknown magnitude of X needs no scale);
//   (2) the leaf solve of each block in FP32 on the CUDA cores, itself a wavefront over 4 x 4
//       sub-blocks of 32 x 32 whose 32 x 32 leaves are eliminated diagonal by diagonal.  The
//       leaf writes X_IJ back (complex128) and refreshes the BF16 planes of X and X^T that the
//       later updates read.
#include <cuda_bf16.h>

#include "lb_internal.cuh"
#include "tc_gemm.cuh"
#include "vecops.cuh"

struct SylvMixed {
    int np = 0, nb = 0;
    __nv_bfloat16* Tp = nullptr;    // 4 x np x np, rows of T (unshifted)
    __nv_bfloat16* Xp = nullptr;    // 4 x np x np, rows of X
    __nv_bfloat16* XTp = nullptr;   // 4 x np x np, rows of X^T
    tc::Maps maps{};                // 0: T, 1: X^T, 2: X
};

namespace {

constexpr int LB = 128;   // wavefront block
constexpr int SB = 32;    // leaf sub-block
constexpr int LEAF_THREADS = 256;
// shared-memory row pitch in complex floats: 130 * 8 B = 1040 B, so that the anti-diagonal
// accesses X[p0 + S - b][q0 + b] of the leaf sweep (stride -pitch + 8 B across lanes) spread over
// the banks (a pitch of 129 would put all 32 lanes on one bank)
constexpr int PITCH = LB + 2;

struct f2 {
    float x, y;
};
__device__ __forceinline__ f2 fmk(float a, float b) { return f2{a, b}; }

__global__ void __launch_bounds__(LEAF_THREADS, 1)
k_sylv_leaf128(const cplx* __restrict__ T, cplx* __restrict__ X, int n, double sh, int wave, int nb,
               __nv_bfloat16* __restrict__ Xp, __nv_bfloat16* __restrict__ XTp, int np) {
    extern __shared__ __align__(16) unsigned char smraw[];
    f2(*Xs)[PITCH] = reinterpret_cast<f2(*)[PITCH]>(smraw);                       // 128 x PITCH
    f2(*Ta)[PITCH] = reinterpret_cast<f2(*)[PITCH]>(smraw + sizeof(f2) * LB * PITCH);
    f2(*Tb)[PITCH] = Ta + SB;                                                     // 32 x PITCH each
    const int t = blockIdx.x + max(0, wave - (nb - 1));
    const int I = nb - 1 - t, J = nb - 1 - (wave - t);
    const int r0 = I * LB, c0 = J * LB;
    const int br = min(LB, n - r0), bc = min(LB, n - c0);
    const int tid = threadIdx.x;
    const float s = (float)sh;

    for (int e = tid; e < LB * LB; e += LEAF_THREADS) {
        const int p = e / LB, q = e % LB;
        cplx v = (p < br && q < bc) ? X[(long long)(r0 + p) * n + c0 + q] : cmake(0, 0);
        Xs[p][q] = fmk((float)v.x, (float)v.y);
    }
    __syncthreads();

    const int PB = (br + SB - 1) / SB, QB = (bc + SB - 1) / SB;
    for (int sw = 0; sw <= (PB - 1) + (QB - 1); ++sw) {
        for (int P = PB - 1; P >= 0; --P) {
            const int Q = (PB - 1 - P) + (QB - 1) - sw;   // (PB-1-P) + (QB-1-Q) = sw
            if (Q < 0 || Q >= QB) continue;
            const int p0 = P * SB, q0 = Q * SB;
            const int sp = min(SB, br - p0), sq = min(SB, bc - q0);
            // stage rows p0.. of A = T_II - sI and rows q0.. of B = T_JJ - sI (columns >= block start)
            for (int e = tid; e < SB * LB; e += LEAF_THREADS) {
                const int a = e / LB, k = e % LB;
                cplx va = (a < sp && k >= p0 && k < br) ? T[(long long)(r0 + p0 + a) * n + r0 + k] : cmake(0, 0);
                cplx vb = (a < sq && k >= q0 && k < bc) ? T[(long long)(c0 + q0 + a) * n + c0 + k] : cmake(0, 0);
                if (k == p0 + a) va.x -= sh;
                if (k == q0 + a) vb.x -= sh;
                Ta[a][k] = fmk((float)va.x, (float)va.y);
                Tb[a][k] = fmk((float)vb.x, (float)vb.y);
            }
            __syncthreads();
            // update from the solved sub-blocks below (rows > p0+32) and to the right (cols > q0+32)
            for (int e = tid; e < SB * SB; e += LEAF_THREADS) {
                const int a = e / SB, b = e % SB;
                if (a >= sp || b >= sq) continue;
                f2 acc = Xs[p0 + a][q0 + b];
                for (int k = p0 + SB; k < br; ++k) {
                    const f2 m = Ta[a][k], x = Xs[k][q0 + b];
                    acc.x -= m.x * x.x - m.y * x.y;
                    acc.y -= m.x * x.y + m.y * x.x;
                }
                for (int k = q0 + SB; k < bc; ++k) {
                    const f2 x = Xs[p0 + a][k], m = Tb[b][k];   // X[a][k] conj(B[b][k])
                    acc.x -= x.x * m.x + x.y * m.y;
                    acc.y -= x.y * m.x - x.x * m.y;
                }
                Xs[p0 + a][q0 + b] = acc;
            }
            __syncthreads();
            // 32 x 32 leaf: A_s X + X B_s^dag = acc, diagonals p + q = S from the corner
            for (int S = (sp - 1) + (sq - 1); S >= 0; --S) {
                for (int e = tid; e < SB * SB; e += LEAF_THREADS) {
                    const int a = e / SB, b = e % SB;
                    if (a < sp && b < sq && a + b == S) {
                        const f2 da = Ta[a][p0 + a], db = Tb[b][q0 + b];
                        const float dr = da.x + db.x, di = da.y - db.y;   // A_aa + conj(B_bb)
                        const float inv = 1.0f / (dr * dr + di * di);
                        const f2 v = Xs[p0 + a][q0 + b];
                        Xs[p0 + a][q0 + b] = fmk((v.x * dr + v.y * di) * inv, (v.y * dr - v.x * di) * inv);
                    }
                }
                __syncthreads();
                for (int e = tid; e < SB * SB; e += LEAF_THREADS) {
                    const int a = e / SB, b = e % SB;
                    if (a < sp && b < sq && a + b < S) {
                        f2 v = Xs[p0 + a][q0 + b];
                        int r = S - b;
                        if (r < sp) {
                            const f2 m = Ta[a][p0 + r], x = Xs[p0 + r][q0 + b];
                            v.x -= m.x * x.x - m.y * x.y;
                            v.y -= m.x * x.y + m.y * x.x;
                        }
                        r = S - a;
                        if (r < sq) {
                            const f2 x = Xs[p0 + a][q0 + r], m = Tb[b][q0 + r];
                            v.x -= x.x * m.x + x.y * m.y;
                            v.y -= x.y * m.x - x.x * m.y;
                        }
                        Xs[p0 + a][q0 + b] = v;
                    }
                }
                __syncthreads();
            }
        }
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

constexpr size_t LEAF_SMEM = sizeof(f2) * LB * PITCH + 2 * sizeof(f2) * SB * PITCH;

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

size_t sylv_mixed_bytes(int n) {
    const size_t np = (size_t)round_up(n, LB);
    return 3 * (4 * np * np * sizeof(__nv_bfloat16) + 256);
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
        k_sylv_leaf128<<<cnt, LEAF_THREADS, LEAF_SMEM, s>>>(h->T, X, h->n, shift, w, nb, m->Xp, m->XTp, m->np);
        lb_note_launch();
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

void sylv_mixed_release(lb_handle_s* h) {
    delete h->sylv;
    h->sylv = nullptr;
}
