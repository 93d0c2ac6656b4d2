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

#include <algorithm>

#include "lb_internal.cuh"
#include "tc_gemm.cuh"
#include "vecops.cuh"

struct SylvMixed {
    int np = 0, nb = 0;
    int sms = 148;                  // multiprocessors of the device (split-K of the wave updates)
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

// barrier of one 128-thread group (named barriers 1..4; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory"); }

constexpr int SB = 32;        // sub-block of the sweep inside a leaf
constexpr int SP = SB + 1;    // pitch of the staged T tiles

// Leaf of one 128 x 128 block (I, J) of the wavefront: A Y + Y B^dag = C with A = T_II - sI,
// B = T_JJ - sI (upper triangular), C already updated by the tensor-core step and held in shared
// memory.  The block is swept in 32 x 32 sub-blocks (p, q) by decreasing p + q, the sub-blocks of
// one p + q in parallel (a 128-thread group each): a sub-block first subtracts its coupling to the
// solved ones, sum_{k>p} A_pk Y_kq + sum_{k>q} Y_pk B_qk^dag (A and B tiles staged from the FP32
// copy of T, Y read in place; 8 outputs per thread), then solves its own 32 x 32 system by
// anti-diagonals,
//   Y_ab = (C_ab - sum_{r>a} A_ar Y_rb - sum_{r>b} Y_ar conj(B_br)) / (A_aa + conj(B_bb)),
// with 4 threads per entry reduced by shuffles, everything in shared memory.
__global__ void __launch_bounds__(LEAF_THREADS, 1)
k_sylv_leaf128(const float2* __restrict__ Tf, const float2* __restrict__ Ttf, int ldf, cplx* __restrict__ X, int n,
               float sh, int wave, int nb, __nv_bfloat16* __restrict__ Xp, __nv_bfloat16* __restrict__ XTp,
               int np) {
    extern __shared__ __align__(16) unsigned char smraw[];
    f2(*Xs)[PITCH] = reinterpret_cast<f2(*)[PITCH]>(smraw);                       // 128 x PITCH
    f2* ta = reinterpret_cast<f2*>(smraw + sizeof(f2) * LB * PITCH);              // 4 groups x 2 x SB x SP
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

    // four groups of 128 threads: the sub-blocks of one sub-anti-diagonal (at most 4) run side by
    // side, each group synchronising on its own named barrier
    const int g = tid >> 7, lt = tid & 127;
    const int tx = lt & 31, ty = lt >> 5;            // rows ty + 4 i (i < 8) of the group's sub-block
    const int slot = lt >> 2, t4 = lt & 3;           // leaf: 32 entries x 4 threads
    f2* ga = ta + g * 2 * SB * SP;                   // the group's two staging tiles
    f2* gb = ga + SB * SP;
    const int nsr = (br + SB - 1) / SB, nsc = (bc + SB - 1) / SB;
    for (int s = (nsr - 1) + (nsc - 1); s >= 0; --s) {
        const int p = max(0, s - (nsc - 1)) + g;
        if (p <= min(s, nsr - 1)) {
            const int q = s - p;
            const int pr = p * SB, qc = q * SB;
            f2 acc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = fmk(0.f, 0.f);
            // sum_{k>p} A_pk Y_kq
            for (int k0 = pr + SB; k0 < br; k0 += SB) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = ty + 4 * i;
                    ga[rr * SP + tx] = (pr + rr < br && k0 + tx < br)
                                           ? f2ld(Tf + (long long)(r0 + pr + rr) * ldf + r0 + k0 + tx) : fmk(0.f, 0.f);
                }
                group_sync(g);
#pragma unroll 4
                for (int k = 0; k < SB; ++k) {
                    const f2 y = Xs[k0 + k][qc + tx];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const f2 m = ga[(ty + 4 * i) * SP + k];
                        acc[i].x += m.x * y.x - m.y * y.y;
                        acc[i].y += m.x * y.y + m.y * y.x;
                    }
                }
                group_sync(g);
            }
            // sum_{k>q} Y_pk B_qk^dag  (gb[k][j] = conj(B[qc + j][k0 + k]): coalesced load, transposed store)
            for (int k0 = qc + SB; k0 < bc; k0 += SB) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = ty + 4 * i;
                    f2 v = (qc + rr < bc && k0 + tx < bc) ? f2ld(Tf + (long long)(c0 + qc + rr) * ldf + c0 + k0 + tx)
                                                          : fmk(0.f, 0.f);
                    v.y = -v.y;
                    gb[tx * SP + rr] = v;
                }
                group_sync(g);
#pragma unroll 4
                for (int k = 0; k < SB; ++k) {
                    const f2 m = gb[k * SP + tx];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const f2 y = Xs[pr + ty + 4 * i][k0 + k];
                        acc[i].x += y.x * m.x - y.y * m.y;
                        acc[i].y += y.x * m.y + y.y * m.x;
                    }
                }
                group_sync(g);
            }
            // right-hand side of the sub-block and its diagonal tiles A_pp, B_qq
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int rr = ty + 4 * i;
                Xs[pr + rr][qc + tx].x -= acc[i].x;
                Xs[pr + rr][qc + tx].y -= acc[i].y;
                ga[rr * SP + tx] = (pr + rr < br && pr + tx < br)
                                       ? f2ld(Tf + (long long)(r0 + pr + rr) * ldf + r0 + pr + tx) : fmk(0.f, 0.f);
                gb[rr * SP + tx] = (qc + rr < bc && qc + tx < bc)
                                       ? f2ld(Tf + (long long)(c0 + qc + rr) * ldf + c0 + qc + tx) : fmk(0.f, 0.f);
            }
            group_sync(g);
            for (int d = 2 * SB - 2; d >= 0; --d) {
                const int alo = max(0, d - (SB - 1)), cnt = min(d, SB - 1) - alo + 1;
                const bool valid = slot < cnt;
                const int a = alo + (valid ? slot : 0), b = d - a;
                // the divisor and the right-hand side do not depend on the sums: read and formed first, off the
                // chain of the step
                const f2 da = ga[a * SP + a], db = gb[b * SP + b];
                const float dr = (da.x - sh) + (db.x - sh), di = da.y - db.y;   // A_aa + conj(B_bb)
                const float inv = 1.0f / (dr * dr + di * di);
                const f2 rhs = Xs[pr + a][qc + b];
                // two partial sums per kind (even / odd term) halve the dependent FMA chains
                f2 acc0 = fmk(0.f, 0.f), acc1 = fmk(0.f, 0.f), acc2 = fmk(0.f, 0.f), acc3 = fmk(0.f, 0.f);
                if (valid) {
                    // the (at most 8) terms of each thread are independent: fully unrolled and predicated
                    // so that their shared-memory loads overlap (this chain of steps sets the leaf's time)
#pragma unroll
                    for (int q = 0; q < SB / 4; ++q) {
                        const int r = a + 1 + t4 + 4 * q;
                        if (r < SB) {
                            const f2 m = ga[a * SP + r], y = Xs[pr + r][qc + b];
                            f2& acc = (q & 1) ? acc2 : acc0;
                            acc.x += m.x * y.x - m.y * y.y;
                            acc.y += m.x * y.y + m.y * y.x;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < SB / 4; ++q) {
                        const int r = b + 1 + t4 + 4 * q;
                        if (r < SB) {
                            const f2 y = Xs[pr + a][qc + r], m = gb[b * SP + r];
                            f2& acc = (q & 1) ? acc3 : acc1;
                            acc.x += y.x * m.x + y.y * m.y;
                            acc.y += y.y * m.x - y.x * m.y;
                        }
                    }
                }
                f2 sum = fmk((acc0.x + acc2.x) + (acc1.x + acc3.x), (acc0.y + acc2.y) + (acc1.y + acc3.y));
                sum.x += __shfl_xor_sync(0xffffffffu, sum.x, 1);
                sum.y += __shfl_xor_sync(0xffffffffu, sum.y, 1);
                sum.x += __shfl_xor_sync(0xffffffffu, sum.x, 2);
                sum.y += __shfl_xor_sync(0xffffffffu, sum.y, 2);
                if (valid && t4 == 0 && pr + a < br && qc + b < bc) {
                    const f2 v = fmk(rhs.x - sum.x, rhs.y - sum.y);
                    Xs[pr + a][qc + b] = fmk((v.x * dr + v.y * di) * inv, (v.y * dr - v.x * di) * inv);
                }
                group_sync(g);
            }
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

constexpr size_t LEAF_SMEM = sizeof(f2) * LB * PITCH + 4 * 2 * sizeof(f2) * SB * SP;

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
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            m->sms = sms;
    }
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
    if (lb_smem_attr((const void*)k_sylv_leaf128, (int)LEAF_SMEM)) return -1;
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
    p.wait_ns = h->tc_wait_ns;
    p.fmt = 1;
    p.nb = nb;
    for (int w = 0; w <= 2 * nb - 2; ++w) {
        const int lo = w - (nb - 1) > 0 ? w - (nb - 1) : 0;
        const int hi = w < nb - 1 ? w : nb - 1;
        const int cnt = hi - lo + 1;
        if (w > 0) {
            // a wave has at most nb blocks: split their K ranges so that the launch fills the SMs
            p.wave = w;
            p.ksplit = std::max(1, std::min(8, m->sms / cnt));
            if (tc_gemm_launch(m->maps, p, cnt, p.ksplit, s)) return -1;
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
