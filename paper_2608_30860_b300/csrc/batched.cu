// Batched steady states of many independent Lindbladians of uneven size (a parameter sweep):
// every instance runs Alg. 4 with complex64 contractions and FP64 anchoring, all instances in one
// persistent launch.
//
//   k_batched_setup  one CTA per instance, FP64: G = -iH - 1/2 sum L^dag L; complex Schur form
//                    G = Q T Q^dag on the device (Householder reduction to Hessenberg form, then
//                    the implicitly shifted single-shift QR algorithm with the unitary accumulated);
//                    L~_j = Q^dag L_j Q; complex64 copies of T and L~; the case-1 test of Theorem 1.
//   k_batched_solve  persistent: each CTA takes instances from an atomic queue (largest n first, so
//                    the tail of the sweep is made of short jobs) and runs Phi-Arnoldi in complex64
//                    (CTA-level GEMMs, anti-diagonal triangular Sylvester solve, modified
//                    Gram-Schmidt applied twice, Ritz value nearest 1 by one warp), then restarts
//                    anchored in FP64 until ||L(rho)||_max < tol in the original basis.
// Both launches (and the queue reset) are captured into a CUDA graph and replayed once.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "lb_internal.cuh"
#include "small_schur.cuh"
#include "vecops.cuh"

namespace bt {

constexpr int BT = 256;   // threads per CTA
constexpr int MB = 32;    // largest Arnoldi cycle in the batched engine
constexpr int GT = 32;    // CTA GEMM tile

struct Inst {
    int n, status;
    int tile;             // complex64 jump-term GEMM tile shape (tgemm_dispatch)
    long long in_off;     // offset (elements) of H / rho in the packed inputs; L at d * in_off
    long long off64;      // FP64 region (complex128 elements)
    long long off32;      // complex64 region
};

struct InstInfo {
    double residual_max, residual_fro;
    int phi_applies, restarts, refine_steps, status;
};

// ------------------------------------------------------------------ complex helpers (float2 / double2)
template <typename C> struct Real;
template <> struct Real<float2> { typedef float T; };
template <> struct Real<double2> { typedef double T; };
template <typename C> __device__ __forceinline__ C cz() { C r; r.x = 0; r.y = 0; return r; }
template <typename C> __device__ __forceinline__ C cm(double a, double b) {
    C r;
    r.x = (typename Real<C>::T)a;
    r.y = (typename Real<C>::T)b;
    return r;
}
template <typename C> __device__ __forceinline__ C ca(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C cs(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmu(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cc(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ void cf(C& c, C a, C b) {
    c.x += a.x * b.x - a.y * b.y;
    c.y += a.x * b.y + a.y * b.x;
}
template <typename C> __device__ __forceinline__ C cdv(C a, C b) {
    const double2 q = cdiv(make_double2(a.x, a.y), make_double2(b.x, b.y));
    return cm<C>(q.x, q.y);
}
// complex64 division kept in FP32 (FP64 instructions are scarce on this part)
template <> __device__ __forceinline__ float2 cdv<float2>(float2 a, float2 b) {
    const float inv = 1.f / (b.x * b.x + b.y * b.y);
    return make_float2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
template <typename C> __device__ __forceinline__ C mk(typename Real<C>::T a, typename Real<C>::T b) {
    C r;
    r.x = a;
    r.y = b;
    return r;
}

// ------------------------------------------------------------------ CTA-level building blocks
// C = alpha op(A) op(B) + beta C  (n x n row-major; op 0 = N, 2 = conjugate transpose);
// sa, sb: GT x (GT+1) shared tiles.  C must not alias A or B.  Structure flags: a_upper -- op(A)
// is upper triangular (k-tiles left of the row tile are skipped); upper_only -- only tiles on or
// above the diagonal are formed (the caller mirrors a Hermitian result).
template <typename C>
__device__ void cta_gemm(const C* A, int opA, const C* B, int opB, C* Cm, int n, C alpha, C beta, int use_beta,
                         C* sa, C* sb, int a_upper = 0, int upper_only = 0) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 x 32
    for (int r0 = 0; r0 < n; r0 += GT) {
        for (int c0 = upper_only ? r0 : 0; c0 < n; c0 += GT) {
            C acc[4] = {cz<C>(), cz<C>(), cz<C>(), cz<C>()};
            for (int k0 = a_upper ? r0 : 0; k0 < n; k0 += GT) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int rr = ty + 8 * i;
                    const int gr = r0 + rr, gk = k0 + tx;
                    C va = cz<C>();
                    if (gr < n && gk < n) va = opA == 0 ? A[(long long)gr * n + gk] : cc(A[(long long)gk * n + gr]);
                    sa[rr * (GT + 1) + tx] = va;
                    const int gk2 = k0 + rr, gc = c0 + tx;
                    C vb = cz<C>();
                    if (gk2 < n && gc < n) vb = opB == 0 ? B[(long long)gk2 * n + gc] : cc(B[(long long)gc * n + gk2]);
                    sb[rr * (GT + 1) + tx] = vb;
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < GT; ++k) {
                    const C b = sb[k * (GT + 1) + tx];
#pragma unroll
                    for (int i = 0; i < 4; ++i) cf(acc[i], sa[(ty + 8 * i) * (GT + 1) + k], b);
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = r0 + ty + 8 * i, c = c0 + tx;
                if (r < n && c < n) {
                    C v = cmu(alpha, acc[i]);
                    if (use_beta) v = ca(v, cmu(beta, Cm[(long long)r * n + c]));
                    Cm[(long long)r * n + c] = v;
                }
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ tunable complex64 CTA GEMM
// C = alpha sum_{s < nseg} A_s op(B_s): A_s = A + s a_seg (M x K row-major), B_s = B + s b_seg (opB 0: K x N
// row-major; opB 2: N x K row-major, taken conjugate-transposed).  Output tile TM x TN per pass, K step KT,
// the BT threads in a (TM/RM) x (TN/RN) grid with an RM x RN register tile each (rows tr + i TM/RM, columns
// tc + j TN/RN: consecutive lanes read consecutive shared-memory columns).  sa: TM x (KT+1), sb: KT x (TN+1)
// complex64 tiles.  The tile shape is the autotuner's choice per instance size.
template <int TM, int TN, int KT, int RM, int RN>
__device__ __forceinline__ void tgemm_c64(const float2* __restrict__ A, long long a_seg, const float2* __restrict__ B,
                                       long long b_seg, int opB, int nseg, float2* __restrict__ Cm, int M, int N, int K,
                                       float alpha, float2* sa, float2* sb) {
    constexpr int RG = TM / RM, CG = TN / RN;
    static_assert(RG * CG == BT, "one register tile per thread");
    const int t = threadIdx.x, tr = t / CG, tc = t % CG;
    for (int r0 = 0; r0 < M; r0 += TM) {
        for (int c0 = 0; c0 < N; c0 += TN) {
            float2 acc[RM][RN];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);
            for (int sg = 0; sg < nseg; ++sg) {
                const float2* As = A + sg * a_seg;
                const float2* Bs = B + sg * b_seg;
                for (int k0 = 0; k0 < K; k0 += KT) {
                    for (int e = t; e < TM * KT; e += BT) {
                        const int rr = e / KT, kk = e % KT, gr = r0 + rr, gk = k0 + kk;
                        sa[rr * (KT + 1) + kk] = (gr < M && gk < K) ? As[(long long)gr * K + gk] : make_float2(0.f, 0.f);
                    }
                    if (opB == 0) {
                        for (int e = t; e < KT * TN; e += BT) {
                            const int kk = e / TN, cc = e % TN, gk = k0 + kk, gc = c0 + cc;
                            sb[kk * (TN + 1) + cc] = (gk < K && gc < N) ? Bs[(long long)gk * N + gc] : make_float2(0.f, 0.f);
                        }
                    } else {
                        for (int e = t; e < KT * TN; e += BT) {
                            const int cc = e / KT, kk = e % KT, gk = k0 + kk, gc = c0 + cc;
                            float2 v = (gk < K && gc < N) ? Bs[(long long)gc * K + gk] : make_float2(0.f, 0.f);
                            v.y = -v.y;
                            sb[kk * (TN + 1) + cc] = v;
                        }
                    }
                    __syncthreads();
#pragma unroll 4
                    for (int k = 0; k < KT; ++k) {
                        float2 av[RM], bv[RN];
#pragma unroll
                        for (int i = 0; i < RM; ++i) av[i] = sa[(tr + RG * i) * (KT + 1) + k];
#pragma unroll
                        for (int j = 0; j < RN; ++j) bv[j] = sb[k * (TN + 1) + tc + CG * j];
#pragma unroll
                        for (int i = 0; i < RM; ++i)
#pragma unroll
                            for (int j = 0; j < RN; ++j) {
                                acc[i][j].x += av[i].x * bv[j].x - av[i].y * bv[j].y;
                                acc[i][j].y += av[i].x * bv[j].y + av[i].y * bv[j].x;
                            }
                    }
                    __syncthreads();
                }
            }
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                    const int r = r0 + tr + RG * i, c = c0 + tc + CG * j;
                    if (r < M && c < N) Cm[(long long)r * N + c] = make_float2(alpha * acc[i][j].x, alpha * acc[i][j].y);
                }
        }
    }
    __syncthreads();
}

// the tile shapes the autotuner chooses from: (TM, TN, KT, RM, RN)
constexpr int NTILES = 4;
__device__ inline void tgemm_dispatch(int tile, const float2* A, long long a_seg, const float2* B, long long b_seg,
                                      int opB, int nseg, float2* Cm, int M, int N, int K, float alpha, float2* sa,
                                      float2* sb) {
    switch (tile) {
        case 1: tgemm_c64<64, 32, 16, 4, 2>(A, a_seg, B, b_seg, opB, nseg, Cm, M, N, K, alpha, sa, sb); break;
        case 2: tgemm_c64<64, 64, 16, 4, 4>(A, a_seg, B, b_seg, opB, nseg, Cm, M, N, K, alpha, sa, sb); break;
        case 3: tgemm_c64<32, 64, 16, 2, 4>(A, a_seg, B, b_seg, opB, nseg, Cm, M, N, K, alpha, sa, sb); break;
        default: tgemm_c64<32, 32, 32, 4, 1>(A, a_seg, B, b_seg, opB, nseg, Cm, M, N, K, alpha, sa, sb); break;
    }
}

// sum over the CTA of a double pair; red: >= 2 * (BT/32) doubles of shared memory
__device__ double2 cta_sum2(double a, double b, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
    __syncthreads();
    double sa = 0.0, sb = 0.0;
    for (int q = 0; q < BT / 32; ++q) { sa += red[2 * q]; sb += red[2 * q + 1]; }
    return make_double2(sa, sb);
}

__device__ double cta_max(double a, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = a;
    __syncthreads();
    double m = red[0];
    for (int q = 1; q < BT / 32; ++q) m = fmax(m, red[q]);
    return m;
}

// <x, y> = sum conj(x) y  (in double)
template <typename C, typename D>
__device__ double2 cta_dot(const C* x, const D* y, long long len, double* red) {
    double re = 0.0, im = 0.0;
    for (long long e = threadIdx.x; e < len; e += BT) {
        const double ax = x[e].x, ay = x[e].y, bx = y[e].x, by = y[e].y;
        re += ax * bx + ay * by;
        im += ax * by - ay * bx;
    }
    return cta_sum2(re, im, red);
}

template <typename C>
__device__ double2 cta_trace(const C* X, int n, double* red) {
    double re = 0.0, im = 0.0;
    for (int i = threadIdx.x; i < n; i += BT) { re += X[(long long)i * n + i].x; im += X[(long long)i * n + i].y; }
    return cta_sum2(re, im, red);
}

// Blocked solve of the triangular Lyapunov equation (T - s) X + X (T - s)^dag = C, in place.
// 32 x 32 blocks (I, J) in decreasing I + J: each block first subtracts the solved coupling
// sum_{K>I} T_IK X_KJ + sum_{K>J} X_IK T_JK^dag (shared-memory tiles, 4 outputs per thread), then
// solves its leaf T_II Y + Y T_JJ^dag = C_IJ in shared memory by anti-diagonals, 8 threads per
// entry.  sa, sb, sc: GT x (GT + 1) shared tiles; entries beyond n are held at zero.
template <typename C>
__device__ void cta_trisylv(const C* T, C* X, int n, double s, C* sa, C* sb, C* sc) {
    typedef typename Real<C>::T R;
    constexpr int P = GT + 1;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int slot = threadIdx.x >> 3, t8 = threadIdx.x & 7;
    const int nb = (n + GT - 1) / GT;
    const R shift2 = (R)(2.0 * s);
    for (int S = 2 * nb - 2; S >= 0; --S) {
        const int Ilo = max(0, S - (nb - 1)), Ihi = min(S, nb - 1);
        for (int I = Ilo; I <= Ihi; ++I) {
            const int J = S - I;
            const int r0 = I * GT, c0 = J * GT;
            C acc[4] = {cz<C>(), cz<C>(), cz<C>(), cz<C>()};
            // T[I rows, k] X[k, J cols] over k >= (I + 1) GT
            for (int k0 = r0 + GT; k0 < n; k0 += GT) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int rr = ty + 8 * i;
                    sa[rr * P + tx] = (r0 + rr < n && k0 + tx < n) ? T[(long long)(r0 + rr) * n + k0 + tx] : cz<C>();
                    sb[rr * P + tx] = (k0 + rr < n && c0 + tx < n) ? X[(long long)(k0 + rr) * n + c0 + tx] : cz<C>();
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < GT; ++k) {
                    const C bv = sb[k * P + tx];
#pragma unroll
                    for (int i = 0; i < 4; ++i) cf(acc[i], sa[(ty + 8 * i) * P + k], bv);
                }
                __syncthreads();
            }
            // X[I rows, k] T[J rows, k]^dag over k >= (J + 1) GT
            for (int k0 = c0 + GT; k0 < n; k0 += GT) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int rr = ty + 8 * i;
                    sa[rr * P + tx] = (r0 + rr < n && k0 + tx < n) ? X[(long long)(r0 + rr) * n + k0 + tx] : cz<C>();
                    // sb[k][j] = conj(T[c0 + j, k0 + k]) (coalesced load, transposed store)
                    sb[tx * P + rr] = (c0 + rr < n && k0 + tx < n) ? cc(T[(long long)(c0 + rr) * n + k0 + tx]) : cz<C>();
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < GT; ++k) {
                    const C bv = sb[k * P + tx];
#pragma unroll
                    for (int i = 0; i < 4; ++i) cf(acc[i], sa[(ty + 8 * i) * P + k], bv);
                }
                __syncthreads();
            }
            // leaf right-hand side and diagonal blocks
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rr = ty + 8 * i;
                const bool in = r0 + rr < n && c0 + tx < n;
                sc[rr * P + tx] = in ? cs(X[(long long)(r0 + rr) * n + c0 + tx], acc[i]) : cz<C>();
                sa[rr * P + tx] = (r0 + rr < n && r0 + tx < n) ? T[(long long)(r0 + rr) * n + r0 + tx] : cz<C>();
                sb[rr * P + tx] = (c0 + rr < n && c0 + tx < n) ? T[(long long)(c0 + rr) * n + c0 + tx] : cz<C>();
            }
            __syncthreads();
            for (int d = 2 * GT - 2; d >= 0; --d) {
                const int alo = max(0, d - (GT - 1)), cnt = min(d, GT - 1) - alo + 1;
                const bool valid = slot < cnt;
                const int a = alo + slot, b = d - a;
                R ax = 0, ay = 0;
                if (valid) {
                    for (int r = a + 1 + t8; r < GT; r += 8) {
                        const C m = sa[a * P + r], x = sc[r * P + b];
                        ax += m.x * x.x - m.y * x.y;
                        ay += m.x * x.y + m.y * x.x;
                    }
                    for (int r = b + 1 + t8; r < GT; r += 8) {
                        const C x = sc[a * P + r], m = sb[b * P + r];
                        ax += x.x * m.x + x.y * m.y;
                        ay += x.y * m.x - x.x * m.y;
                    }
                }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    ax += __shfl_xor_sync(0xffffffffu, ax, o);
                    ay += __shfl_xor_sync(0xffffffffu, ay, o);
                }
                if (valid && t8 == 0 && r0 + a < n && c0 + b < n) {
                    const C ta = sa[a * P + a], tb = sb[b * P + b];
                    const C den = mk<C>(ta.x + tb.x - shift2, ta.y - tb.y);
                    sc[a * P + b] = cdv(cs(sc[a * P + b], mk<C>(ax, ay)), den);
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rr = ty + 8 * i;
                if (r0 + rr < n && c0 + tx < n) X[(long long)(r0 + rr) * n + c0 + tx] = sc[rr * P + tx];
            }
            __syncthreads();
        }
    }
}

// barrier of one 128-thread group (named barriers 1, 2; 0 is __syncthreads)
__device__ __forceinline__ void group_sync128(int g) { asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory"); }

// The same blocked solve in complex64 with the blocks of one anti-diagonal shared by two 128-thread
// groups (even and odd I), each with its own three staging tiles (tiles: 6 x GT x (GT + 1)):
// 8 outputs per thread in the updates, 4 threads per entry in the 32 x 32 leaves.
__device__ void cta_trisylv_c64(const float2* T, float2* X, int n, float2* tiles) {
    constexpr int P = GT + 1;
    const int g = threadIdx.x >> 7, lt = threadIdx.x & 127;
    const int tx = lt & 31, ty = lt >> 5;
    const int slot = lt >> 2, t4 = lt & 3;
    float2* sa = tiles + g * 3 * GT * P;
    float2* sb = sa + GT * P;
    float2* sc = sb + GT * P;
    const int nb = (n + GT - 1) / GT;
    for (int S = 2 * nb - 2; S >= 0; --S) {
        const int Ilo = max(0, S - (nb - 1)), Ihi = min(S, nb - 1);
        for (int I = Ilo + g; I <= Ihi; I += 2) {
            const int J = S - I;
            const int r0 = I * GT, c0 = J * GT;
            float2 acc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
            for (int k0 = r0 + GT; k0 < n; k0 += GT) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = ty + 4 * i;
                    sa[rr * P + tx] = (r0 + rr < n && k0 + tx < n) ? T[(long long)(r0 + rr) * n + k0 + tx] : make_float2(0.f, 0.f);
                    sb[rr * P + tx] = (k0 + rr < n && c0 + tx < n) ? X[(long long)(k0 + rr) * n + c0 + tx] : make_float2(0.f, 0.f);
                }
                group_sync128(g);
#pragma unroll 4
                for (int k = 0; k < GT; ++k) {
                    const float2 bv = sb[k * P + tx];
#pragma unroll
                    for (int i = 0; i < 8; ++i) cf(acc[i], sa[(ty + 4 * i) * P + k], bv);
                }
                group_sync128(g);
            }
            for (int k0 = c0 + GT; k0 < n; k0 += GT) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = ty + 4 * i;
                    sa[rr * P + tx] = (r0 + rr < n && k0 + tx < n) ? X[(long long)(r0 + rr) * n + k0 + tx] : make_float2(0.f, 0.f);
                    sb[tx * P + rr] = (c0 + rr < n && k0 + tx < n) ? cc(T[(long long)(c0 + rr) * n + k0 + tx]) : make_float2(0.f, 0.f);
                }
                group_sync128(g);
#pragma unroll 4
                for (int k = 0; k < GT; ++k) {
                    const float2 bv = sb[k * P + tx];
#pragma unroll
                    for (int i = 0; i < 8; ++i) cf(acc[i], sa[(ty + 4 * i) * P + k], bv);
                }
                group_sync128(g);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int rr = ty + 4 * i;
                const bool in = r0 + rr < n && c0 + tx < n;
                sc[rr * P + tx] = in ? cs(X[(long long)(r0 + rr) * n + c0 + tx], acc[i]) : make_float2(0.f, 0.f);
                sa[rr * P + tx] = (r0 + rr < n && r0 + tx < n) ? T[(long long)(r0 + rr) * n + r0 + tx] : make_float2(0.f, 0.f);
                sb[rr * P + tx] = (c0 + rr < n && c0 + tx < n) ? T[(long long)(c0 + rr) * n + c0 + tx] : make_float2(0.f, 0.f);
            }
            group_sync128(g);
            for (int d = 2 * GT - 2; d >= 0; --d) {
                const int alo = max(0, d - (GT - 1)), cnt = min(d, GT - 1) - alo + 1;
                const bool valid = slot < cnt;
                const int a = alo + slot, b = d - a;
                float ax = 0.f, ay = 0.f;
                if (valid) {
                    // independent terms, fully unrolled and predicated so that the loads overlap
#pragma unroll
                    for (int q = 0; q < GT / 4; ++q) {
                        const int r = a + 1 + t4 + 4 * q;
                        if (r < GT) {
                            const float2 m = sa[a * P + r], x = sc[r * P + b];
                            ax += m.x * x.x - m.y * x.y;
                            ay += m.x * x.y + m.y * x.x;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < GT / 4; ++q) {
                        const int r = b + 1 + t4 + 4 * q;
                        if (r < GT) {
                            const float2 x = sc[a * P + r], m = sb[b * P + r];
                            ax += x.x * m.x + x.y * m.y;
                            ay += x.y * m.x - x.x * m.y;
                        }
                    }
                }
                ax += __shfl_xor_sync(0xffffffffu, ax, 1);
                ay += __shfl_xor_sync(0xffffffffu, ay, 1);
                ax += __shfl_xor_sync(0xffffffffu, ax, 2);
                ay += __shfl_xor_sync(0xffffffffu, ay, 2);
                if (valid && t4 == 0 && r0 + a < n && c0 + b < n) {
                    const float2 ta = sa[a * P + a], tb = sb[b * P + b];
                    const float2 den = make_float2(ta.x + tb.x, ta.y - tb.y);
                    sc[a * P + b] = cdv(cs(sc[a * P + b], make_float2(ax, ay)), den);
                }
                group_sync128(g);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int rr = ty + 4 * i;
                if (r0 + rr < n && c0 + tx < n) X[(long long)(r0 + rr) * n + c0 + tx] = sc[rr * P + tx];
            }
            group_sync128(g);
        }
        __syncthreads();
    }
}

// complex Schur form of A (n x n, global, FP64) in place, unitary accumulated in Z (= Q):
// Householder reduction to Hessenberg form, then implicitly shifted single-shift QR.
// hv: n scratch (global); shared: red, sh (rotation / flags).  Returns 1 on a stall.
__device__ int cta_schur(cplx* A, cplx* Z, int n, cplx* hv, double* red, cplx* shc, double* shd, int* shi) {
    const int tid = threadIdx.x;
    const double eps = 2.220446049250313e-16;
    for (long long e = tid; e < (long long)n * n; e += BT) Z[e] = cmake((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        double p = 0.0;
        for (int i = k + 1 + tid; i < n; i += BT) p += cabs2(A[(long long)i * n + k]);
        const double xn2 = cta_sum2(p, 0.0, red).x;
        const cplx x0 = A[(long long)(k + 1) * n + k];
        const double xn = sqrt(xn2);
        if (xn == 0.0 || xn2 - cabs2(x0) <= 1e-300 * xn2) { __syncthreads(); continue; }
        const double ax0 = sqrt(cabs2(x0));
        const cplx ph = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : cmake(1.0, 0.0);
        const cplx alpha = cscale(ph, -xn);
        for (int i = k + 1 + tid; i < n; i += BT) {
            cplx v = A[(long long)i * n + k];
            if (i == k + 1) v = csub(v, alpha);
            hv[i] = v;
        }
        __syncthreads();
        p = 0.0;
        for (int i = k + 1 + tid; i < n; i += BT) p += cabs2(hv[i]);
        const double vn = sqrt(cta_sum2(p, 0.0, red).x);
        for (int i = k + 1 + tid; i < n; i += BT) hv[i] = cscale(hv[i], 1.0 / vn);
        __syncthreads();
        for (int j = k + tid; j < n; j += BT) {        // A <- (I - 2 v v^H) A
            cplx s = cmake(0, 0);
            for (int i = k + 1; i < n; ++i) cfma(s, cconj(hv[i]), A[(long long)i * n + j]);
            for (int i = k + 1; i < n; ++i)
                A[(long long)i * n + j] = csub(A[(long long)i * n + j], cscale(cmul(hv[i], s), 2.0));
        }
        __syncthreads();
        for (int i = tid; i < n; i += BT) {             // A <- A (I - 2 v v^H), Z <- Z (I - 2 v v^H)
            cplx sa = cmake(0, 0), sz = cmake(0, 0);
            for (int j = k + 1; j < n; ++j) {
                cfma(sa, A[(long long)i * n + j], hv[j]);
                cfma(sz, Z[(long long)i * n + j], hv[j]);
            }
            for (int j = k + 1; j < n; ++j) {
                A[(long long)i * n + j] = csub(A[(long long)i * n + j], cscale(cmul(sa, cconj(hv[j])), 2.0));
                Z[(long long)i * n + j] = csub(Z[(long long)i * n + j], cscale(cmul(sz, cconj(hv[j])), 2.0));
            }
        }
        __syncthreads();
        for (int i = k + 2 + tid; i < n; i += BT) A[(long long)i * n + k] = cmake(0, 0);
        __syncthreads();
    }
    int hi = n - 1, iter = 0, total = 0;
    const int max_total = 30 * n;
    while (hi > 0) {
        if (total >= max_total) return 1;
        if (tid == 0) {
            int l = hi;
            while (l > 0) {
                const double sub = sqrt(cabs2(A[(long long)l * n + l - 1]));
                const double dg = sqrt(cabs2(A[(long long)l * n + l])) + sqrt(cabs2(A[(long long)(l - 1) * n + l - 1]));
                if (sub <= eps * dg || sub < 1e-300) break;
                --l;
            }
            if (l > 0) A[(long long)l * n + l - 1] = cmake(0, 0);
            shi[0] = l;
        }
        __syncthreads();
        const int l = shi[0];
        __syncthreads();
        if (l == hi) { --hi; iter = 0; continue; }
        if (tid == 0) {
            cplx mu;
            const cplx dd = A[(long long)hi * n + hi];
            if (iter == 10 || iter == 20) {
                const double s = fabs(A[(long long)hi * n + hi - 1].x) + fabs(A[(long long)hi * n + hi - 1].y);
                mu = cadd(dd, cmake(0.75 * s, 0.0));
            } else {
                const cplx a = A[(long long)(hi - 1) * n + hi - 1], b = A[(long long)(hi - 1) * n + hi];
                const cplx c = A[(long long)hi * n + hi - 1];
                const cplx half = cscale(csub(a, dd), 0.5);
                const cplx disc = csqrt_d(cadd(cmul(half, half), cmul(b, c)));
                const cplx mid = cscale(cadd(a, dd), 0.5);
                const cplx m1 = cadd(mid, disc), m2 = csub(mid, disc);
                mu = (cabs2(csub(m1, dd)) <= cabs2(csub(m2, dd))) ? m1 : m2;
            }
            shc[1] = mu;
        }
        __syncthreads();
        const cplx mu = shc[1];
        for (int k = l; k < hi; ++k) {
            if (tid == 0) {
                cplx x, y;
                if (k == l) { x = csub(A[(long long)l * n + l], mu); y = A[(long long)(l + 1) * n + l]; }
                else { x = A[(long long)k * n + k - 1]; y = A[(long long)(k + 1) * n + k - 1]; }
                double c; cplx s;
                givens(x, y, c, s);
                shd[0] = c;
                shc[0] = s;
            }
            __syncthreads();
            const double c = shd[0];
            const cplx s = shc[0];
            for (int j = (k == l ? l : k - 1) + tid; j < n; j += BT) {
                const cplx a = A[(long long)k * n + j], b = A[(long long)(k + 1) * n + j];
                A[(long long)k * n + j] = cadd(cscale(a, c), cmul(s, b));
                A[(long long)(k + 1) * n + j] = csub(cscale(b, c), cmul(cconj(s), a));
            }
            __syncthreads();
            const int rmax = min(k + 2, hi);
            for (int i = tid; i <= rmax; i += BT) {
                const cplx a = A[(long long)i * n + k], b = A[(long long)i * n + k + 1];
                A[(long long)i * n + k] = cadd(cscale(a, c), cmul(b, cconj(s)));
                A[(long long)i * n + k + 1] = csub(cscale(b, c), cmul(a, s));
            }
            for (int i = tid; i < n; i += BT) {
                const cplx a = Z[(long long)i * n + k], b = Z[(long long)i * n + k + 1];
                Z[(long long)i * n + k] = cadd(cscale(a, c), cmul(b, cconj(s)));
                Z[(long long)i * n + k + 1] = csub(cscale(b, c), cmul(a, s));
            }
            __syncthreads();
            if (k > l && tid == 0) A[(long long)(k + 1) * n + k - 1] = cmake(0, 0);
            __syncthreads();
        }
        ++iter;
        ++total;
    }
    for (long long e = tid; e < (long long)n * n; e += BT)
        if (e / n > e % n) A[e] = cmake(0, 0);
    __syncthreads();
    return 0;
}

// ------------------------------------------------------------------ per-instance storage
constexpr int PK = 6;    // Ritz values nearest 1 carried across a restart (the first is the iterate)

struct View {
    int n, d, tile;
    cplx *G, *Q, *T, *Lt, *S1, *S2, *S3, *S4, *S5, *S6, *hv;   // FP64
    float2 *Tf, *Ltf, *V, *Wa, *Ub, *Z1, *Pf;                 // complex64
};

__host__ __device__ inline long long f64_elems(int n, int d) { return (long long)(9 + d) * n * n + n; }
__host__ __device__ inline long long f32_elems(int n, int d) {
    return (long long)(1 + d + (MB + 1) + 2 * (PK - 1) + 1 + d) * n * n;
}

__device__ View make_view(const Inst& in, int d, cplx* a64, float2* a32) {
    View v;
    const int n = in.n;
    const long long nn = (long long)n * n;
    v.n = n;
    v.d = d;
    v.tile = in.tile;
    cplx* p = a64 + in.off64;
    v.G = p; p += nn;
    v.Q = p; p += nn;
    v.T = p; p += nn;
    v.Lt = p; p += d * nn;
    v.S1 = p; p += nn;
    v.S2 = p; p += nn;
    v.S3 = p; p += nn;
    v.S4 = p; p += nn;
    v.S5 = p; p += nn;
    v.S6 = p; p += nn;
    v.hv = p;
    float2* q = a32 + in.off32;
    v.Tf = q; q += nn;
    v.Ltf = q; q += d * nn;
    v.V = q; q += (MB + 1) * nn;
    v.Wa = q; q += (PK - 1) * nn;
    v.Ub = q; q += (PK - 1) * nn;
    v.Z1 = q; q += nn;
    v.Pf = q;
    return v;
}

struct Shared {
    cplx ga[GT * (GT + 1)];
    cplx gb[GT * (GT + 1)];
    cplx gc[GT * (GT + 1)];
    double red[64];
    cplx hm[(MB + 1) * MB];      // projected matrix V^dag Phi V, column-major, ld MB + 1
    cplx ssA[MB * (MB + 1)], ssZ[MB * (MB + 1)], ssV[MB * (MB + 1)];
    cplx ev[MB], zs[MB * MB], hvv[MB + 1];
    cplx hb[MB + 1];             // block dot products
    float2 hbf[MB + 1];          // the same in FP32
    float2 zsf[MB * MB];         // carried Schur vectors' coefficients in FP32
    cplx alpha[MB + 1];          // <v0, V_i> in FP64 (v0 the FP64 anchor, V_i the stored complex64 vector)
    double nu[MB + 1];           // || V_i - alpha_i v0 ||
    cplx shc[4];
    double shd[4];
    int shi[4];
};

// -------------------------------------------------------------- complex64 operators of one instance
// y = alpha * sum_j L~_j Z L~_j^dag  (complex64, Pf scratch)
__device__ void jump32(const View& v, const float2* Zin, float2* y, float alpha, Shared& sm) {
    const long long nn = (long long)v.n * v.n;
    float2* sa = reinterpret_cast<float2*>(sm.ga);
    float2* sb = reinterpret_cast<float2*>(sm.gb);
    if (v.tile == 0) {
        // shape 0: the general CTA GEMM, one product per jump (P_j = L~_j Z, then y += alpha P_j L~_j^dag)
        for (int j = 0; j < v.d; ++j)
            cta_gemm(v.Ltf + j * nn, 0, Zin, 0, v.Pf + j * nn, v.n, make_float2(1.f, 0.f), make_float2(0.f, 0.f), 0,
                     sa, sb);
        for (int j = 0; j < v.d; ++j)
            cta_gemm(v.Pf + j * nn, 0, v.Ltf + j * nn, 2, y, v.n, make_float2(alpha, 0.f), make_float2(1.f, 0.f),
                     j > 0, sa, sb);
        return;
    }
    // (1) [P_1; ..; P_d] = [L~_1; ..; L~_d] Z  (one stacked product, M = d n)
    tgemm_dispatch(v.tile, v.Ltf, 0, Zin, 0, 0, 1, v.Pf, v.d * v.n, v.n, v.n, 1.f, sa, sb);
    // (2) y = alpha sum_j P_j L~_j^dag  (the sum over j inside one accumulation)
    tgemm_dispatch(v.tile, v.Pf, nn, v.Ltf, nn, 2, v.d, y, v.n, v.n, v.n, alpha, sa, sb);
}

// w = Phi(x) = -K~(S~^{-1} x) in complex64 (Z1 scratch)
__device__ void phi32(const View& v, const float2* x, float2* w, Shared& sm) {
    const long long nn = (long long)v.n * v.n;
    for (long long e = threadIdx.x; e < nn; e += BT) v.Z1[e] = x[e];
    __syncthreads();
    cta_trisylv_c64(v.Tf, v.Z1, v.n, reinterpret_cast<float2*>(sm.ga));
    jump32(v, v.Z1, w, -1.f, sm);
}

// sm.hb[i] = <V_i, w>, i < cnt: one warp per vector, FP32 products and partial sums
__device__ void multidot32(const float2* V, long long nn, int cnt, const float2* w, Shared& sm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < cnt; i += BT / 32) {
        const float2* vi = V + i * nn;
        float re = 0.f, im = 0.f;
        for (long long e = lane; e < nn; e += 32) {
            const float2 a = vi[e], b = w[e];
            re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));
            im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            sm.hb[i] = cmake(re, im);
            sm.hbf[i] = make_float2(re, im);
        }
    }
    __syncthreads();
}

// ||x||^2 of a complex64 vector (FP32 partial sums per thread, CTA reduction in FP64)
__device__ double norm2_32(const float2* x, long long nn, Shared& sm) {
    float acc = 0.f;
    for (long long e = threadIdx.x; e < nn; e += BT) acc = fmaf(x[e].x, x[e].x, fmaf(x[e].y, x[e].y, acc));
    return cta_sum2((double)acc, 0.0, sm.red).x;
}

// w <- w - sum_{i<cnt} hb[i] V_i (complex64)
__device__ void multiaxpy32(const float2* V, long long nn, int cnt, float2* w, const Shared& sm) {
    for (long long e = threadIdx.x; e < nn; e += BT) {
        float2 acc = w[e];
        for (int i = 0; i < cnt; ++i) {
            const float2 a = V[i * nn + e];
            const float2 h = sm.hbf[i];
            acc.x -= h.x * a.x - h.y * a.y;
            acc.y -= h.x * a.y + h.y * a.x;
        }
        w[e] = acc;
    }
    __syncthreads();
}

// the stored complex64 vector V_i stands for v~_i = (V_i - alpha_i v0) / nu_i, exactly orthogonal
// to the FP64 anchor v0: alpha_i = <v0, V_i>, nu_i^2 = <V_i, V_i> - |alpha_i|^2, both in FP64
__device__ void anchor_coeffs(const cplx* v0, const float2* x, long long nn, int slot, Shared& sm) {
    double ar = 0.0, ai = 0.0, s2 = 0.0;
    for (long long e = threadIdx.x; e < nn; e += BT) {
        const cplx a = v0[e];
        const double bx = x[e].x, by = x[e].y;
        ar += a.x * bx + a.y * by;
        ai += a.x * by - a.y * bx;
        s2 += bx * bx + by * by;
    }
    const double2 al = cta_sum2(ar, ai, sm.red);
    const double nn2 = cta_sum2(s2, 0.0, sm.red).x;
    if (threadIdx.x == 0) {
        sm.alpha[slot] = al;
        sm.nu[slot] = sqrt(fmax(nn2 - cabs2(al), 0.0));
    }
    __syncthreads();
}

// X <- (X / Tr X + (X / Tr X)^dag) / 2, then divided by its (real) trace; tmp: n x n scratch
__device__ void herm_normalize(cplx* X, cplx* tmp, int n, double* red) {
    const long long nn = (long long)n * n;
    double2 tr = cta_trace(X, n, red);
    for (long long e = threadIdx.x; e < nn; e += BT) tmp[e] = cdiv(X[e], tr);
    __syncthreads();
    for (long long e = threadIdx.x; e < nn; e += BT) {
        const long long i = e / n, j = e % n;
        const cplx a = tmp[e], b = tmp[j * n + i];
        X[e] = cmake(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
    __syncthreads();
    tr = cta_trace(X, n, red);
    for (long long e = threadIdx.x; e < nn; e += BT) X[e] = cscale(X[e], 1.0 / tr.x);
    __syncthreads();
}

// lower triangle of a Hermitian matrix from its upper triangle
template <typename C>
__device__ void mirror_lower(C* X, int n) {
    const long long nn = (long long)n * n;
    for (long long e = threadIdx.x; e < nn; e += BT) {
        const long long i = e / n, j = e % n;
        if (i > j) X[e] = cc(X[j * n + i]);
    }
    __syncthreads();
}

// ------------------------------------------------------------------ kernels
__global__ void __launch_bounds__(BT, 1)
k_batched_setup(Inst* insts, int count, int d, const cplx* __restrict__ Hin,
                const cplx* __restrict__ Lin, cplx* a64, float2* a32, InstInfo* infos) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Shared& sm = *reinterpret_cast<Shared*>(smraw);
    const int idx = blockIdx.x;
    if (idx >= count) return;
    Inst in = insts[idx];
    const View v = make_view(in, d, a64, a32);
    const int n = v.n;
    const long long nn = (long long)n * n;
    const cplx* H = Hin + in.in_off;
    const cplx* L = Lin + (long long)d * in.in_off;
    // G = -iH - 1/2 sum_j L_j^dag L_j
    for (long long e = threadIdx.x; e < nn; e += BT) v.G[e] = cmake(H[e].y, -H[e].x);
    __syncthreads();
    for (int j = 0; j < d; ++j)
        cta_gemm(L + j * nn, 2, L + j * nn, 0, v.G, n, cmake(-0.5, 0), cmake(1, 0), 1, sm.ga, sm.gb);
    // Schur form: A (in T) <- G, Q accumulated
    for (long long e = threadIdx.x; e < nn; e += BT) v.T[e] = v.G[e];
    __syncthreads();
    const int stalled = cta_schur(v.T, v.Q, n, v.hv, sm.red, sm.shc, sm.shd, sm.shi);
    // case 1 of Theorem 1 (an eigenvalue of G on the imaginary axis) against ||G||_F
    double mre = 1e300, g2 = 0.0;
    for (int i = threadIdx.x; i < n; i += BT) mre = fmin(mre, fabs(v.T[(long long)i * n + i].x));
    for (long long e = threadIdx.x; e < nn; e += BT) g2 += cabs2(v.G[e]);
    const double gf = sqrt(cta_sum2(g2, 0.0, sm.red).x);
    mre = -cta_max(-mre, sm.red);
    const int case1 = mre <= 1e3 * 2.220446049250313e-16 * gf;
    // L~_j = Q^dag L_j Q
    for (int j = 0; j < d; ++j) {
        cta_gemm(v.Q, 2, L + j * nn, 0, v.S1, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb);
        cta_gemm(v.S1, 0, v.Q, 0, v.Lt + j * nn, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb);
    }
    for (long long e = threadIdx.x; e < nn; e += BT) v.Tf[e] = make_float2((float)v.T[e].x, (float)v.T[e].y);
    for (long long e = threadIdx.x; e < d * nn; e += BT)
        v.Ltf[e] = make_float2((float)v.Lt[e].x, (float)v.Lt[e].y);
    if (threadIdx.x == 0) {
        Inst* wi = insts + idx;
        wi->status = case1 ? LB_S_SINGULAR : (stalled ? LB_SOLVER_ERROR : LB_OK);
        InstInfo inf;
        inf.residual_max = inf.residual_fro = -1.0;
        inf.phi_applies = inf.restarts = inf.refine_steps = 0;
        inf.status = wi->status;
        infos[idx] = inf;
    }
}

// One restart cycle of the augmented Phi-Arnoldi on one instance.
//   Basis: v0 (FP64, S4) -- the normalised iterate xi (phase 1) or the anchor S~ rho~ (phase 2) --,
//   then the carried Schur vectors (Ub), the remainder of Phi v0, and Arnoldi vectors; every vector
//   after v0 is stored in complex64 and used as v~_i = (V_i - alpha_i v0) / nu_i, exactly orthogonal
//   to v0, so the FP64 iterate never mixes with complex64 rounding.  Phi v0 is w0 (FP64, S5).
//   The projected matrix V^dag Phi V (sm.hm) is reduced to ordered Schur form (one warp); the new
//   iterate is the orthogonal projection of e0 on the Schur vectors of the eigenvalues within
//   1e-6 of the one nearest 1 (a numerically degenerate cluster keeps its current mixture), the
//   next PK - 1 Schur vectors are carried.  Returns the Ritz residual estimate; xi (S1) is updated.
__device__ double aug_cycle(const View& v, int m, int& nU, int& applies, Shared& sm, double& theta_abs) {
    const int n = v.n;
    const long long nn = (long long)n * n;
    cplx* v0 = v.S4;
    cplx* w0 = v.S5;
    for (int e = threadIdx.x; e < (MB + 1) * MB; e += BT) sm.hm[e] = cmake(0, 0);
    if (threadIdx.x == 0) { sm.alpha[0] = cmake(0, 0); sm.nu[0] = 1.0; }
    for (long long e = threadIdx.x; e < nn; e += BT) v.V[e] = make_float2((float)v0[e].x, (float)v0[e].y);
    __syncthreads();
    // carried vectors: orthogonalise (complex64, twice) against the basis so far, then exactly against v0
    int q = 1;
    for (int s = 0; s < nU; ++s) {
        float2* x = v.V + q * nn;
        for (long long e = threadIdx.x; e < nn; e += BT) x[e] = v.Ub[s * nn + e];
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            multidot32(v.V, nn, q, x, sm);
            multiaxpy32(v.V, nn, q, x, sm);
        }
        const double xn = sqrt(fmax(norm2_32(x, nn, sm), 0.0));
        if (!(xn > 1e-3)) continue;
        for (long long e = threadIdx.x; e < nn; e += BT) { x[e].x /= (float)xn; x[e].y /= (float)xn; }
        __syncthreads();
        anchor_coeffs(v0, x, nn, q, sm);
        phi32(v, x, v.Wa + (q - 1) * nn, sm);
        ++applies;
        ++q;
    }
    // remainder of w0 = Phi v0 after projection on v0 and the carried vectors (FP64, twice)
    for (int pass = 0; pass < 2; ++pass) {
        double pr = 0.0, pi = 0.0;
        for (long long e = threadIdx.x; e < nn; e += BT) {
            const cplx a = v0[e], b = w0[e];
            pr += a.x * b.x + a.y * b.y;
            pi += a.x * b.y - a.y * b.x;
        }
        const double2 c0 = cta_sum2(pr, pi, sm.red);
        for (int i = 1; i < q; ++i) {
            const float2* x = v.V + i * nn;
            double dr = 0.0, di = 0.0;
            for (long long e = threadIdx.x; e < nn; e += BT) {
                const double ax = x[e].x, ay = x[e].y;
                const cplx b = w0[e];
                dr += ax * b.x + ay * b.y;
                di += ax * b.y - ay * b.x;
            }
            const double2 di2 = cta_sum2(dr, di, sm.red);
            // <v~_i, w0> = (<V_i, w0> - conj(alpha_i) <v0, w0>) / nu_i
            if (threadIdx.x == 0) sm.hb[i] = cscale(csub(di2, cmul(cconj(sm.alpha[i]), c0)), 1.0 / sm.nu[i]);
        }
        if (threadIdx.x == 0) sm.hb[0] = c0;
        __syncthreads();
        // w0 -= c0 v0 + sum_i c_i v~_i  =  w0 - (c0 - sum_i c_i alpha_i / nu_i) v0 - sum_i (c_i / nu_i) V_i
        cplx cv0 = sm.hb[0];
        for (int i = 1; i < q; ++i) cv0 = csub(cv0, cscale(cmul(sm.hb[i], sm.alpha[i]), 1.0 / sm.nu[i]));
        for (long long e = threadIdx.x; e < nn; e += BT) {
            cplx acc = csub(w0[e], cmul(cv0, v0[e]));
            for (int i = 1; i < q; ++i) {
                const float2 x = v.V[i * nn + e];
                acc = csub(acc, cmul(cscale(sm.hb[i], 1.0 / sm.nu[i]), make_double2(x.x, x.y)));
            }
            w0[e] = acc;
        }
        if (threadIdx.x == 0)
            for (int i = 0; i < q; ++i) sm.hm[i] = cadd(sm.hm[i], sm.hb[i]);
        __syncthreads();
    }
    const double b0 = sqrt(fmax(cta_dot(w0, w0, nn, sm.red).x, 0.0));
    int kk = q;
    if (b0 > 1e-300 && q < m) {
        if (threadIdx.x == 0) sm.hm[q] = cmake(b0, 0.0);
        float2* x = v.V + q * nn;
        for (long long e = threadIdx.x; e < nn; e += BT)
            x[e] = make_float2((float)(w0[e].x / b0), (float)(w0[e].y / b0));
        __syncthreads();
        anchor_coeffs(v0, x, nn, q, sm);
        kk = q + 1;
        // Arnoldi continuation: columns j = q .. m-1
        for (int j = q; j < m; ++j) {
            float2* w = v.V + (j + 1) * nn;
            phi32(v, v.V + j * nn, w, sm);
            ++applies;
            const double wn = sqrt(fmax(norm2_32(w, nn, sm), 0.0));
            for (int pass = 0; pass < 2; ++pass) {
                multidot32(v.V, nn, j + 1, w, sm);
                multiaxpy32(v.V, nn, j + 1, w, sm);
                if (threadIdx.x == 0)
                    for (int i = 0; i <= j; ++i) sm.hm[j * (MB + 1) + i] = cadd(sm.hm[j * (MB + 1) + i], sm.hb[i]);
                __syncthreads();
            }
            const double beta = sqrt(fmax(norm2_32(w, nn, sm), 0.0));
            if (threadIdx.x == 0) sm.hm[j * (MB + 1) + j + 1] = cmake(beta, 0.0);
            __syncthreads();
            if (!(beta > 1e-6 * wn) || j + 1 == m) break;
            for (long long e = threadIdx.x; e < nn; e += BT) { w[e].x /= (float)beta; w[e].y /= (float)beta; }
            __syncthreads();
            anchor_coeffs(v0, w, nn, j + 1, sm);
            kk = j + 2;
        }
    }
    // columns of the carried vectors: <V_i, Phi V_c> for every basis vector
    for (int c = 1; c < q; ++c) {
        multidot32(v.V, nn, kk, v.Wa + (c - 1) * nn, sm);
        if (threadIdx.x == 0)
            for (int i = 0; i < kk; ++i) sm.hm[c * (MB + 1) + i] = sm.hb[i];
        __syncthreads();
    }
    // ordered Schur form of the kk x kk projected matrix
    if (threadIdx.x < 32)
        small_schur_warp(sm.hm, MB + 1, kk, 0, 2, PK < kk ? PK : kk, sm.ev, nullptr, nullptr, sm.zs, nullptr, sm.ssA,
                         sm.ssZ, sm.ssV, sm.hvv, sm.shc[2], sm.shd[2]);
    __syncthreads();
    const int npk = PK < kk ? PK : kk;
    const double d0 = sqrt(cabs2(csub(sm.ev[0], cmake(1, 0))));
    int cl = 1;
    while (cl < npk && sqrt(cabs2(csub(sm.ev[cl], cmake(1, 0)))) <= d0 + 1e-6) ++cl;
    theta_abs = sqrt(cabs2(sm.ev[0]));
    // y = Z_c Z_c^dag e0 (column-major Z, ld kk), normalised; Ritz residual estimate
    if (threadIdx.x == 0) {
        double yn = 0.0, zl = 0.0;
        for (int t = 0; t < kk; ++t) {
            cplx acc = cmake(0, 0);
            for (int s = 0; s < cl; ++s) cfma(acc, sm.zs[s * kk + t], cconj(sm.zs[s * kk]));
            sm.hvv[t] = acc;
            yn += cabs2(acc);
        }
        for (int s = 0; s < cl; ++s) zl += cabs2(sm.zs[s * kk + kk - 1]);
        for (int t = 0; t < kk; ++t) sm.hvv[t] = cscale(sm.hvv[t], 1.0 / sqrt(yn));
        const int jl = kk - 1;
        sm.shd[0] = sqrt(cabs2(sm.hm[jl * (MB + 1) + kk])) * sqrt(zl);
        // v0 coefficient of xi = sum_t y_t v~_t
        cplx c0 = sm.hvv[0];
        for (int t = 1; t < kk; ++t) c0 = csub(c0, cscale(cmul(sm.hvv[t], sm.alpha[t]), 1.0 / sm.nu[t]));
        sm.shc[0] = c0;
    }
    __syncthreads();
    const double rr = sm.shd[0];
    const cplx c0 = sm.shc[0];
    cplx* xi = v.S1;
    for (long long e = threadIdx.x; e < nn; e += BT) {
        cplx acc = cmul(c0, v0[e]);
        for (int t = 1; t < kk; ++t) {
            const float2 x = v.V[t * nn + e];
            acc = cadd(acc, cmul(cscale(sm.hvv[t], 1.0 / sm.nu[t]), make_double2(x.x, x.y)));
        }
        xi[e] = acc;
    }
    __syncthreads();
    const double2 tr = cta_trace(xi, n, sm.red);
    for (long long e = threadIdx.x; e < nn; e += BT) xi[e] = cdiv(xi[e], tr);
    // carried Schur vectors 1 .. npk-1 (complex64)
    nU = npk - 1;
    for (int e = threadIdx.x; e < npk * kk; e += BT) sm.zsf[e] = make_float2((float)sm.zs[e].x, (float)sm.zs[e].y);
    __syncthreads();
    for (long long e = threadIdx.x; e < nn; e += BT) {
        for (int s = 1; s < npk; ++s) {
            float ax = 0.f, ay = 0.f;
            for (int t = 0; t < kk; ++t) {
                const float2 x = v.V[t * nn + e];
                const float2 z = sm.zsf[s * kk + t];
                ax += z.x * x.x - z.y * x.y;
                ay += z.x * x.y + z.y * x.x;
            }
            v.Ub[(s - 1) * nn + e] = make_float2(ax, ay);
        }
    }
    __syncthreads();
    return rr;
}

// Persistent solve: each CTA takes instances from the queue.  Per instance
//   phase 1  complex64 cycles (aug_cycle, v0 = xi / ||xi||, Phi v0 in complex64) from I / n while
//            the Ritz residual keeps falling and is above 1e-5 |theta|;
//   phase 2  cycles anchored in FP64: rho~ = S~^{-1} xi (FP64 triangular solve), hermitised,
//            trace 1; v0 = S~ rho~ / ||.||, Phi v0 = -K~ rho~ / ||.|| (FP64), so only the
//            correction carries complex64 rounding.  The Schur-coordinate residual L~ rho~ =
//            S~ rho~ + K~ rho~ comes with the anchor; once it is below the trigger, rho = Q rho~
//            Q^dag and L(rho) are formed in FP64 in the original basis and the instance stops
//            when ||L(rho)||_max < tol.
__global__ void __launch_bounds__(BT, 1)
k_batched_solve(const Inst* __restrict__ insts, const int* __restrict__ order, int count, int d,
                const cplx* __restrict__ Lin, cplx* __restrict__ rho_out, cplx* a64, float2* a32, int* queue,
                double tol, int m, int max_restarts, InstInfo* infos) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Shared& sm = *reinterpret_cast<Shared*>(smraw);
    __shared__ int job;
    while (true) {
        if (threadIdx.x == 0) job = atomicAdd(queue, 1);
        __syncthreads();
        const int qj = job;
        __syncthreads();
        if (qj >= count) break;
        const int idx = order[qj];
        const Inst in = insts[idx];
        if (in.status != LB_OK) continue;
        const View v = make_view(in, d, a64, a32);
        const int n = v.n;
        const long long nn = (long long)n * n;
        const cplx* L = Lin + (long long)d * in.in_off;
        cplx* rho = rho_out + in.in_off;
        int applies = 0, restarts = 0, anchors = 0, nU = 0;
        cplx* xi = v.S1;
        for (long long e = threadIdx.x; e < nn; e += BT)
            xi[e] = cmake((e / n) == (e % n) ? 1.0 / n : 0.0, 0.0);
        __syncthreads();
        // ---- phase 1
        double best = 1e300, th = 1.0;
        int since = 0;
        for (int rs = 0; rs < max_restarts; ++rs) {
            ++restarts;
            const double xn = sqrt(cta_dot(xi, xi, nn, sm.red).x);
            for (long long e = threadIdx.x; e < nn; e += BT) v.S4[e] = cscale(xi[e], 1.0 / xn);
            __syncthreads();
            for (long long e = threadIdx.x; e < nn; e += BT) v.V[e] = make_float2((float)v.S4[e].x, (float)v.S4[e].y);
            __syncthreads();
            phi32(v, v.V, v.V + nn, sm);
            ++applies;
            for (long long e = threadIdx.x; e < nn; e += BT) v.S5[e] = make_double2(v.V[nn + e].x, v.V[nn + e].y);
            __syncthreads();
            const double rr = aug_cycle(v, m, nU, applies, sm, th);
            if (rr < 0.7 * best) { best = rr; since = 0; }
            else ++since;
            if (rr < 1e-5 * th || since >= 3) break;
        }
        // ---- phase 2
        cplx* rt = v.S2;
        double trigger = tol, rmax = 1e300, rfro = 1e300;
        bool done = false;
        for (int rs = 0; rs < max_restarts; ++rs) {
            ++anchors;
            for (long long e = threadIdx.x; e < nn; e += BT) rt[e] = xi[e];
            __syncthreads();
            cta_trisylv(v.T, rt, n, 0.0, sm.ga, sm.gb, sm.gc);
            herm_normalize(rt, v.S3, n, sm.red);
            // S4 = T rho~ + rho~ T^dag, S5 = K~ rho~, Schur-coordinate residual S4 + S5
            cta_gemm(v.T, 0, rt, 0, v.S3, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb, 1, 0);
            for (long long e = threadIdx.x; e < nn; e += BT) {
                const long long i = e / n, j = e % n;
                v.S4[e] = cadd(v.S3[e], cconj(v.S3[j * n + i]));
            }
            for (int j = 0; j < d; ++j) {
                cta_gemm(v.Lt + j * nn, 0, rt, 0, v.S3, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb);
                cta_gemm(v.S3, 0, v.Lt + j * nn, 2, v.S5, n, cmake(1, 0), cmake(1, 0), j > 0, sm.ga, sm.gb, 0, 1);
            }
            mirror_lower(v.S5, n);
            double mx = 0.0;
            for (long long e = threadIdx.x; e < nn; e += BT) mx = fmax(mx, cabs2(cadd(v.S4[e], v.S5[e])));
            const double rs_max = sqrt(cta_max(mx, sm.red));
            if (rs_max < trigger || rs + 1 == max_restarts) {
                // rho = Q rho~ Q^dag (hermitised, trace 1) and L(rho) in the original basis
                cta_gemm(v.Q, 0, rt, 0, v.S3, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb);
                cta_gemm(v.S3, 0, v.Q, 2, rho, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb);
                herm_normalize(rho, v.S3, n, sm.red);
                // L(rho) = G rho + (G rho)^dag + sum_j L_j rho L_j^dag (rho Hermitian; upper triangle, mirrored)
                cta_gemm(v.G, 0, rho, 0, v.S6, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb);
                for (long long e = threadIdx.x; e < nn; e += BT) {
                    const long long i = e / n, j = e % n;
                    v.S3[e] = cadd(v.S6[e], cconj(v.S6[j * n + i]));
                }
                __syncthreads();
                for (int j = 0; j < d; ++j) {
                    cta_gemm(L + j * nn, 0, rho, 0, v.S6, n, cmake(1, 0), cmake(0, 0), 0, sm.ga, sm.gb);
                    cta_gemm(v.S6, 0, L + j * nn, 2, v.S3, n, cmake(1, 0), cmake(1, 0), 1, sm.ga, sm.gb, 0, 1);
                }
                mirror_lower(v.S3, n);
                double m2 = 0.0, s2 = 0.0;
                for (long long e = threadIdx.x; e < nn; e += BT) {
                    const double a2 = cabs2(v.S3[e]);
                    m2 = fmax(m2, a2);
                    s2 += a2;
                }
                rmax = sqrt(cta_max(m2, sm.red));
                rfro = sqrt(cta_sum2(s2, 0.0, sm.red).x);
                if (rmax < tol) { done = true; break; }
                trigger *= 0.1;
            }
            if (rs + 1 == max_restarts) break;
            ++restarts;
            const double nx = sqrt(cta_dot(v.S4, v.S4, nn, sm.red).x);
            for (long long e = threadIdx.x; e < nn; e += BT) {
                v.S4[e] = cscale(v.S4[e], 1.0 / nx);
                v.S5[e] = cscale(v.S5[e], -1.0 / nx);
            }
            __syncthreads();
            aug_cycle(v, m, nU, applies, sm, th);
        }
        if (threadIdx.x == 0) {
            InstInfo inf;
            inf.residual_max = rmax;
            inf.residual_fro = rfro;
            inf.phi_applies = applies;
            inf.restarts = restarts;
            inf.refine_steps = anchors;
            inf.status = done ? LB_OK : LB_NOT_CONVERGED;
            infos[idx] = inf;
        }
        __syncthreads();
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// the private stream, events and graph of one call, released on every return path (an unfinished
// capture is ended and its graph dropped)
struct CallResources {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool capturing = false;
    ~CallResources() {
        if (capturing) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (cs) cudaStreamDestroy(cs);
    }
};

struct Plan {
    std::vector<Inst> insts;
    std::vector<int> order;
    long long n64 = 0, n32 = 0, packed = 0;
    size_t bytes = 0, off_inst = 0, off_order = 0, off_info = 0, off_queue = 0, off64 = 0, off32 = 0;
};

bool make_plan(int count, const int* n, int d, Plan& p, const int* tiles = nullptr) {
    p.insts.resize(count);
    long long in_off = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 2 || n[i] > 256) return false;
        Inst& in = p.insts[i];
        in.n = n[i];
        in.status = 0;
        in.tile = tiles ? tiles[std::min((n[i] - 1) / 16, LB_TILE_BUCKETS - 1)] : 0;
        if (in.tile < 0 || in.tile >= NTILES) return false;
        in.in_off = in_off;
        in.off64 = p.n64;
        in.off32 = p.n32;
        in_off += (long long)n[i] * n[i];
        p.n64 += f64_elems(n[i], d);
        p.n32 += f32_elems(n[i], d);
    }
    p.packed = in_off;
    p.order.resize(count);
    std::iota(p.order.begin(), p.order.end(), 0);
    std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) { return n[a] > n[b]; });   // LPT
    size_t off = 0;
    p.off_inst = off; off = align256(off + count * sizeof(Inst));
    p.off_order = off; off = align256(off + count * sizeof(int));
    p.off_info = off; off = align256(off + count * sizeof(InstInfo));
    p.off_queue = off; off = align256(off + sizeof(int));
    p.off64 = off; off = align256(off + (size_t)p.n64 * sizeof(cplx));
    p.off32 = off; off = align256(off + (size_t)p.n32 * sizeof(float2));
    p.bytes = off;
    return true;
}

// ------------------------------------------------------------------ tile autotuner
// Deterministic complex64 operands for the tuner (values in [-1, 1], no randomness needed for timing).
__global__ void k_tune_fill(float2* buf, long long len) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
        buf[e] = make_float2(__sinf(0.37f * (float)(e % 9973)), __cosf(0.11f * (float)(e % 7919)));
}

// One CTA per synthetic instance of size n: reps complex64 jump terms y = -sum_j L_j (Z) L_j^dag with tile
// shape `tile`, exactly as jump32 forms them.  Slice of CTA b: L (d n^2), Z (n^2), P (d n^2), y (n^2).
__global__ void __launch_bounds__(BT, 1) k_tune_jump(int tile, int n, int d, float2* buf, int reps) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Shared& sm = *reinterpret_cast<Shared*>(smraw);
    const long long nn = (long long)n * n;
    float2* L = buf + (long long)blockIdx.x * (2 * d + 2) * nn;
    float2* Z = L + d * nn;
    float2* P = Z + nn;
    float2* y = P + d * nn;
    float2* sa = reinterpret_cast<float2*>(sm.ga);
    float2* sb = reinterpret_cast<float2*>(sm.gb);
    for (int r = 0; r < reps; ++r) {
        if (tile == 0) {
            for (int j = 0; j < d; ++j)
                cta_gemm(L + j * nn, 0, Z, 0, P + j * nn, n, make_float2(1.f, 0.f), make_float2(0.f, 0.f), 0, sa, sb);
            for (int j = 0; j < d; ++j)
                cta_gemm(P + j * nn, 0, L + j * nn, 2, y, n, make_float2(-1.f, 0.f), make_float2(1.f, 0.f), j > 0, sa,
                         sb);
            continue;
        }
        tgemm_dispatch(tile, L, 0, Z, 0, 0, 1, P, d * n, n, n, 1.f, sa, sb);
        tgemm_dispatch(tile, P, nn, L, nn, 2, d, y, n, n, n, -1.f, sa, sb);
    }
}

}  // namespace bt

namespace {
int tune_instances() {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm;
}
}  // namespace

extern "C" size_t lindblad_batched_tune_workspace_bytes(int d, int nmax) {
    if (d < 1 || nmax < 2 || nmax > 256) return 0;
    return (size_t)tune_instances() * (2 * d + 2) * (size_t)nmax * nmax * sizeof(float2);
}

extern "C" lb_status lindblad_batched_tune(int d, int nmax, void* workspace, size_t ws_bytes, int* tiles_out,
                                           float* us_out, void* stream) {
    if (d < 1 || nmax < 2 || nmax > 256 || !workspace || !tiles_out) return LB_INVALID_ARG;
    const size_t need = lindblad_batched_tune_workspace_bytes(d, nmax);
    if (ws_bytes < need) return LB_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    const int smem = (int)sizeof(bt::Shared);
    if (lb_smem_attr((const void*)bt::k_tune_jump, smem)) return LB_CUDA_ERROR;
    const int ninst = tune_instances();
    float2* buf = static_cast<float2*>(workspace);
    bt::k_tune_fill<<<1184, 256, 0, s>>>(buf, (long long)(need / sizeof(float2)));
    lb_note_launch();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LB_CHECK_CUDA(cudaEventCreate(&e0));
    LB_CHECK_CUDA(cudaEventCreate(&e1));
    lb_status st = LB_OK;
    for (int b = 0; b < LB_TILE_BUCKETS && st == LB_OK; ++b) {
        // the bucket's largest size (the one that sets its cost), capped at nmax
        const int n = std::min(16 * (b + 1), nmax);
        if (b > 0 && n == std::min(16 * b, nmax)) {   // past nmax: the same size as the previous bucket
            tiles_out[b] = tiles_out[b - 1];
            if (us_out)
                for (int t = 0; t < bt::NTILES; ++t) us_out[b * bt::NTILES + t] = us_out[(b - 1) * bt::NTILES + t];
            continue;
        }
        // about 2e8 complex MACs per instance per timed launch, at least one jump term
        const double macs = 2.0 * d * (double)n * n * n;
        const int reps = (int)std::max(1.0, std::min(64.0, 2e8 / macs));
        float best = 0.f;
        int bi = 0;
        for (int t = 0; t < bt::NTILES; ++t) {
            bt::k_tune_jump<<<ninst, bt::BT, smem, s>>>(t, n, d, buf, 1);   // warm-up
            lb_note_launch();
            cudaEventRecord(e0, s);
            bt::k_tune_jump<<<ninst, bt::BT, smem, s>>>(t, n, d, buf, reps);
            lb_note_launch();
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = LB_CUDA_ERROR; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const float us = 1000.f * ms / reps;   // one jump term per instance, all instances side by side
            if (us_out) us_out[b * bt::NTILES + t] = us;
            if (t == 0 || us < best) { best = us; bi = t; }
        }
        tiles_out[b] = bi;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return LB_CUDA_ERROR;
    return st;
}

extern "C" size_t lindblad_batched_workspace_bytes(int count, const int* n, int d, const lb_opts* opts) {
    (void)opts;
    if (count < 1 || !n || d < 1) return 0;
    bt::Plan p;
    if (!bt::make_plan(count, n, d, p)) return 0;
    return p.bytes;
}

extern "C" lb_status steady_state_batched(int count, const int* n, int d, const void* H_dev, const void* L_dev,
                                          void* rho_dev, void* workspace, size_t ws_bytes, const lb_opts* opts,
                                          lb_info* infos, void* stream) {
    if (count < 1 || !n || d < 1 || !H_dev || !L_dev || !rho_dev || !workspace) return LB_INVALID_ARG;
    lb_opts o;
    lb_default_opts(&o);
    if (opts) o = *opts;
    const int m = std::min(std::max(o.krylov_m, bt::PK + 2), bt::MB);
    bt::Plan p;
    if (!bt::make_plan(count, n, d, p, o.batched_tiles)) return LB_INVALID_ARG;
    if (p.bytes > ws_bytes) return LB_WORKSPACE_TOO_SMALL;
    char* ws = static_cast<char*>(workspace);
    bt::Inst* d_inst = reinterpret_cast<bt::Inst*>(ws + p.off_inst);
    int* d_order = reinterpret_cast<int*>(ws + p.off_order);
    bt::InstInfo* d_info = reinterpret_cast<bt::InstInfo*>(ws + p.off_info);
    int* d_queue = reinterpret_cast<int*>(ws + p.off_queue);
    cplx* a64 = reinterpret_cast<cplx*>(ws + p.off64);
    float2* a32 = reinterpret_cast<float2*>(ws + p.off32);
    cudaStream_t user = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const int smem = (int)sizeof(bt::Shared);
    if (lb_smem_attr((const void*)bt::k_batched_setup, smem) || lb_smem_attr((const void*)bt::k_batched_solve, smem))
        return LB_CUDA_ERROR;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    LB_CHECK_CUDA(cudaMemcpyAsync(d_inst, p.insts.data(), count * sizeof(bt::Inst), cudaMemcpyHostToDevice, user));
    LB_CHECK_CUDA(cudaMemcpyAsync(d_order, p.order.data(), count * sizeof(int), cudaMemcpyHostToDevice, user));
    // the launches run as one captured graph on a private stream ordered after the caller's stream
    bt::CallResources r;
    LB_CHECK_CUDA(cudaStreamCreateWithFlags(&r.cs, cudaStreamNonBlocking));
    LB_CHECK_CUDA(cudaEventCreateWithFlags(&r.ev0, cudaEventDisableTiming));
    LB_CHECK_CUDA(cudaEventCreateWithFlags(&r.ev1, cudaEventDisableTiming));
    LB_CHECK_CUDA(cudaEventRecord(r.ev0, user));
    LB_CHECK_CUDA(cudaStreamWaitEvent(r.cs, r.ev0, 0));
    cudaStream_t cs = r.cs;
    LB_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    r.capturing = true;
    LB_CHECK_CUDA(cudaMemsetAsync(d_queue, 0, sizeof(int), cs));
    bt::k_batched_setup<<<count, bt::BT, smem, cs>>>(d_inst, count, d, (const cplx*)H_dev, (const cplx*)L_dev, a64,
                                                      a32, d_info);
    lb_note_launch();
    const int grid = std::min(count, nsm);
    bt::k_batched_solve<<<grid, bt::BT, smem, cs>>>(d_inst, d_order, count, d, (const cplx*)L_dev, (cplx*)rho_dev, a64, a32, d_queue,
                                                     o.tol, m, o.max_restarts, d_info);
    lb_note_launch();
    r.capturing = false;
    LB_CHECK_CUDA(cudaStreamEndCapture(cs, &r.graph));
    LB_CHECK_CUDA(cudaGraphInstantiate(&r.exec, r.graph, 0));
    LB_CHECK_CUDA(cudaGraphLaunch(r.exec, cs));
    LB_CHECK_CUDA(cudaEventRecord(r.ev1, cs));
    LB_CHECK_CUDA(cudaStreamWaitEvent(user, r.ev1, 0));
    std::vector<bt::InstInfo> hi(count);
    LB_CHECK_CUDA(cudaMemcpyAsync(hi.data(), d_info, count * sizeof(bt::InstInfo), cudaMemcpyDeviceToHost, user));
    LB_CHECK_CUDA(cudaStreamSynchronize(user));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    lb_status worst = LB_OK;
    for (int i = 0; i < count; ++i) {
        if (infos) {
            lb_info& inf = infos[i];
            std::memset(&inf, 0, sizeof(inf));
            inf.status = hi[i].status;
            inf.residual_max = hi[i].residual_max;
            inf.residual_fro = hi[i].residual_fro;
            inf.phi_applies = hi[i].phi_applies;
            inf.restarts = hi[i].restarts;
            inf.refine_steps = hi[i].refine_steps;
            inf.solve_ms = ms;
        }
        if (hi[i].status < 0 && worst >= 0) worst = (lb_status)hi[i].status;
        else if (hi[i].status > 0 && worst == LB_OK) worst = (lb_status)hi[i].status;
    }
    return worst;
}
