// Mixed-precision triangular Lyapunov solve (T - sI) X + X (T - sI)^dag = C in Schur
// coordinates (the Bartels-Stewart back substitution of App. A.1.1), for the tensor-core path.
//
// Blocks of 128 x 128 are swept by anti-diagonals from the bottom-right corner.  Per
// anti-diagonal w two launches:
//   (1) the left-looking update of every block (I, J) on w,
//         C_IJ -= sum_{K>I} T_IK X_KJ + sum_{L>J} X_IL T_JL^dag,
//       one tcgen05 CTA per block (tc_gemm.cu, wavefront mode, BF16 hi/lo operands -- BF16 keeps
//       FP32's exponent range, so the unknown magnitude of X needs no scale);
//   (2) the leaf solve of each block in FP32 on the CUDA cores, itself blocked: 32 x 32
//       sub-blocks by anti-diagonals, each a small GEMM update plus a 32 x 32 anti-diagonal sweep.  The leaf writes X_IJ back (complex128)
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
constexpr int LEAF_THREADS = 512;
// shared-memory row pitch of the block in complex floats: a column walk of 16 rows (the leaf's
// per-entry split) lands on 16 distinct bank pairs (10 r mod 32)
constexpr int PITCH = LB + 5;

struct f2 {
    float x, y;
};
__device__ __forceinline__ f2 fmk(float a, float b) { return f2{a, b}; }

__device__ __forceinline__ f2 f2ld(const float2* p) { const float2 v = __ldg(p); return fmk(v.x, v.y); }

constexpr int SB = 32;        // sub-block of the sweep inside a leaf
constexpr int SP = SB + 1;    // pitch of the staged T tiles

// Leaf of one 128 x 128 block (I, J) of the wavefront: A Y + Y B^dag = C with A = T_II - sI,
// B = T_JJ - sI (upper triangular), C already updated by the tensor-core step and held in shared
// memory.  The block is swept in 32 x 32 sub-blocks (p, q) by decreasing p + q: a sub-block first
// subtracts its coupling to the solved ones, sum_{k>p} A_pk Y_kq + sum_{k>q} Y_pk B_qk^dag (A and B
// tiles staged from the FP32 copy of T, Y read in place; 2 outputs per thread), then solves its own
// 32 x 32 system by anti-diagonals,
//   Y_ab = (C_ab - sum_{r>a} A_ar Y_rb - sum_{r>b} Y_ar conj(B_br)) / (A_aa + conj(B_bb)),
// with 16 threads per entry reduced by shuffles, everything in shared memory.
__global__ void __launch_bounds__(LEAF_THREADS, 1)
k_sylv_leaf128(const float2* __restrict__ Tf, const float2* __restrict__ Ttf, int ldf, cplx* __restrict__ X, int n,
               float sh, int wave, int nb, __nv_bfloat16* __restrict__ Xp, __nv_bfloat16* __restrict__ XTp,
               int np) {
    extern __shared__ __align__(16) unsigned char smraw[];
    f2(*Xs)[PITCH] = reinterpret_cast<f2(*)[PITCH]>(smraw);                       // 128 x PITCH
    f2* ta = reinterpret_cast<f2*>(smraw + sizeof(f2) * LB * PITCH);              // SB x SP
    f2* tb = ta + SB * SP;                                                         // SB x SP
    const int t = blockIdx.x + max(0, wave - (nb - 1));
    const int I = nb - 1 - t, J = nb - 1 - (wave - t);
    const int r0 = I * LB, c0 = J * LB;
    const int br = min(LB, n - r0), bc = min(LB, n - c0);
    const int tid = threadIdx.x;
    (void)Ttf;

    for (int e = tid; e < LB * LB; e += LEAF_THREADS) {
        const int p = e / LB, q = e % LB;
        const cplx v = (p < br && q < bc) ? X[(long long)(r0 + p) * n + c0 + q] : cmake(0, 0);
        Xs[p][q] = fmk((float)v.x, (float)v.y);
    }
    __syncthreads();

    const int tx = tid & 31, ty = tid >> 5;          // 16 x 32: rows ty and ty + 16 of a sub-block
    const int slot = tid >> 4, t16 = tid & 15;       // leaf: 32 entries x 16 threads
    const int nsr = (br + SB - 1) / SB, nsc = (bc + SB - 1) / SB;
    for (int s = (nsr - 1) + (nsc - 1); s >= 0; --s) {
        for (int p = max(0, s - (nsc - 1)); p <= min(s, nsr - 1); ++p) {
            const int q = s - p;
            const int pr = p * SB, qc = q * SB;
            f2 acc0 = fmk(0.f, 0.f), acc1 = fmk(0.f, 0.f);
            // sum_{k>p} A_pk Y_kq
            for (int k0 = pr + SB; k0 < br; k0 += SB) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int rr = ty + 16 * i;
                    ta[rr * SP + tx] = (pr + rr < br && k0 + tx < br)
                                           ? f2ld(Tf + (long long)(r0 + pr + rr) * ldf + r0 + k0 + tx) : fmk(0.f, 0.f);
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < SB; ++k) {
                    const f2 y = Xs[k0 + k][qc + tx];
                    const f2 m0 = ta[ty * SP + k], m1 = ta[(ty + 16) * SP + k];
                    acc0.x += m0.x * y.x - m0.y * y.y;
                    acc0.y += m0.x * y.y + m0.y * y.x;
                    acc1.x += m1.x * y.x - m1.y * y.y;
                    acc1.y += m1.x * y.y + m1.y * y.x;
                }
                __syncthreads();
            }
            // sum_{k>q} Y_pk B_qk^dag  (tb[k][j] = conj(B[qc + j][k0 + k]): coalesced load, transposed store)
            for (int k0 = qc + SB; k0 < bc; k0 += SB) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int rr = ty + 16 * i;
                    f2 v = (qc + rr < bc && k0 + tx < bc) ? f2ld(Tf + (long long)(c0 + qc + rr) * ldf + c0 + k0 + tx)
                                                          : fmk(0.f, 0.f);
                    v.y = -v.y;
                    tb[tx * SP + rr] = v;
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < SB; ++k) {
                    const f2 m = tb[k * SP + tx];
                    const f2 y0 = Xs[pr + ty][k0 + k], y1 = Xs[pr + ty + 16][k0 + k];
                    acc0.x += y0.x * m.x - y0.y * m.y;
                    acc0.y += y0.x * m.y + y0.y * m.x;
                    acc1.x += y1.x * m.x - y1.y * m.y;
                    acc1.y += y1.x * m.y + y1.y * m.x;
                }
                __syncthreads();
            }
            // right-hand side of the sub-block and its diagonal tiles A_pp, B_qq
            Xs[pr + ty][qc + tx].x -= acc0.x;
            Xs[pr + ty][qc + tx].y -= acc0.y;
            Xs[pr + ty + 16][qc + tx].x -= acc1.x;
            Xs[pr + ty + 16][qc + tx].y -= acc1.y;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int rr = ty + 16 * i;
                ta[rr * SP + tx] = (pr + rr < br && pr + tx < br)
                                       ? f2ld(Tf + (long long)(r0 + pr + rr) * ldf + r0 + pr + tx) : fmk(0.f, 0.f);
                tb[rr * SP + tx] = (qc + rr < bc && qc + tx < bc)
                                       ? f2ld(Tf + (long long)(c0 + qc + rr) * ldf + c0 + qc + tx) : fmk(0.f, 0.f);
            }
            __syncthreads();
            for (int d = 2 * SB - 2; d >= 0; --d) {
                const int alo = max(0, d - (SB - 1)), cnt = min(d, SB - 1) - alo + 1;
                const bool valid = slot < cnt;
                const int a = alo + slot, b = d - a;
                f2 acc = fmk(0.f, 0.f);
                if (valid) {
                    for (int r = a + 1 + t16; r < SB; r += 16) {
                        const f2 m = ta[a * SP + r], y = Xs[pr + r][qc + b];
                        acc.x += m.x * y.x - m.y * y.y;
                        acc.y += m.x * y.y + m.y * y.x;
                    }
                    for (int r = b + 1 + t16; r < SB; r += 16) {
                        const f2 y = Xs[pr + a][qc + r], m = tb[b * SP + r];
                        acc.x += y.x * m.x + y.y * m.y;
                        acc.y += y.y * m.x - y.x * m.y;
                    }
                }
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                }
                if (valid && t16 == 0 && pr + a < br && qc + b < bc) {
                    const f2 da = ta[a * SP + a], db = tb[b * SP + b];
                    const float dr = (da.x - sh) + (db.x - sh), di = da.y - db.y;   // A_aa + conj(B_bb)
                    const float inv = 1.0f / (dr * dr + di * di);
                    const f2 v = fmk(Xs[pr + a][qc + b].x - acc.x, Xs[pr + a][qc + b].y - acc.y);
                    Xs[pr + a][qc + b] = fmk((v.x * dr + v.y * di) * inv, (v.y * dr - v.x * di) * inv);
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

constexpr size_t LEAF_SMEM = sizeof(f2) * LB * PITCH + 2 * sizeof(f2) * SB * SP;

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
