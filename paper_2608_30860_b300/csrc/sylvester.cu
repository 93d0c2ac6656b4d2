// Triangular Lyapunov solve  A X + X A^dag = C,  A = T - s I upper triangular  (App. A.1.1).
//
// Bartels-Stewart on the Schur form G = Q T Q^dag reduces (lam - S)^{-1} to this triangular
// equation with s = lam/2 (the shift T -> T - lam/2 I).  Written block-wise with blocks of
// b x b, block X_IJ depends on X_KJ (K > I) and X_IL (L > J) only:
//
//   A_II X_IJ + X_IJ A_JJ^dag = C_IJ - sum_{K>I} T_IK X_KJ - sum_{L>J} X_IL T_JL^dag
//
// so all blocks on one anti-diagonal (I + J = const) are independent.  One launch per
// anti-diagonal (2 nb - 1 launches, swept from the bottom-right corner); one CTA per block
// does the left-looking update (a b x b x (2n - ...) product of already-solved strips) and
// then the b x b leaf solve in shared memory, itself an anti-diagonal sweep in which each
// solved diagonal is immediately eliminated from the pending entries (right-looking, two
// complex FMAs per entry per step).  All arithmetic in FP64.  X overwrites C in place.
#include "common.cuh"

namespace {

constexpr int SB = 32;          // block size
constexpr int SYL_THREADS = 256;

__global__ void __launch_bounds__(SYL_THREADS)
trisylv_f64_wave(const cplx* __restrict__ T, cplx* __restrict__ X, int n, cplx s, int wave, int nb) {
    // dynamic shared memory: three (SB x SB+1) tiles; the update phase stages strip tiles in
    // the first two, the leaf phase keeps A_II, A_JJ and X_IJ in all three.
    extern __shared__ __align__(16) unsigned char syl_smem[];
    typedef cplx Tile[SB + 1];
    Tile* Sa = reinterpret_cast<Tile*>(syl_smem);
    Tile* Sb = Sa + SB;
    Tile* Xs = Sb + SB;
    Tile* Ta = Sa;
    Tile* Tb = Sb;

    // block (I, J) on this anti-diagonal: (nb-1-I) + (nb-1-J) = wave
    const int lo = max(0, wave - (nb - 1));
    const int t = lo + blockIdx.x;                 // t = nb-1-I
    const int I = nb - 1 - t;
    const int J = nb - 1 - (wave - t);
    if (I < 0 || J < 0 || I >= nb || J >= nb) return;
    const int r0 = I * SB, c0 = J * SB;
    const int br = min(SB, n - r0), bc = min(SB, n - c0);
    const int tid = threadIdx.x;

    // owned entries: e = tid + 256*k, p = e / 32, q = e % 32
    cplx acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int e = tid + SYL_THREADS * k, p = e / SB, q = e % SB;
        acc[k] = (p < br && q < bc) ? X[(long long)(r0 + p) * n + c0 + q] : cmake(0.0, 0.0);
    }

    // left-looking update 1: acc -= sum_{K>I} T[I,K] X[K,J]
    for (int K = I + 1; K < nb; ++K) {
        const int k0 = K * SB, bk = min(SB, n - k0);
        for (int e = tid; e < SB * SB; e += SYL_THREADS) {
            int p = e / SB, q = e % SB;
            Sa[p][q] = (p < br && q < bk) ? T[(long long)(r0 + p) * n + k0 + q] : cmake(0.0, 0.0);
            Sb[p][q] = (p < bk && q < bc) ? X[(long long)(k0 + p) * n + c0 + q] : cmake(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int e = tid + SYL_THREADS * k, p = e / SB, q = e % SB;
            cplx a = acc[k];
#pragma unroll 8
            for (int r = 0; r < SB; ++r) {
                cplx m = Sa[p][r], x = Sb[r][q];
                a.x -= m.x * x.x - m.y * x.y;
                a.y -= m.x * x.y + m.y * x.x;
            }
            acc[k] = a;
        }
        __syncthreads();
    }
    // left-looking update 2: acc -= sum_{L>J} X[I,L] T[J,L]^dag
    for (int L = J + 1; L < nb; ++L) {
        const int l0 = L * SB, bl = min(SB, n - l0);
        for (int e = tid; e < SB * SB; e += SYL_THREADS) {
            int p = e / SB, q = e % SB;
            Sa[p][q] = (p < br && q < bl) ? X[(long long)(r0 + p) * n + l0 + q] : cmake(0.0, 0.0);
            Sb[p][q] = (p < bc && q < bl) ? T[(long long)(c0 + p) * n + l0 + q] : cmake(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int e = tid + SYL_THREADS * k, p = e / SB, q = e % SB;
            cplx a = acc[k];
#pragma unroll 8
            for (int r = 0; r < SB; ++r) {
                cplx x = Sa[p][r], m = Sb[q][r];     // X[p][r] * conj(T[q][r])
                a.x -= x.x * m.x + x.y * m.y;
                a.y -= x.y * m.x - x.x * m.y;
            }
            acc[k] = a;
        }
        __syncthreads();
    }

    // leaf: A_II X + X A_JJ^dag = acc
    for (int e = tid; e < SB * SB; e += SYL_THREADS) {
        int p = e / SB, q = e % SB;
        cplx va = (p < br && q < br) ? T[(long long)(r0 + p) * n + r0 + q] : cmake(0.0, 0.0);
        cplx vb = (p < bc && q < bc) ? T[(long long)(c0 + p) * n + c0 + q] : cmake(0.0, 0.0);
        if (p == q) { va = csub(va, s); vb = csub(vb, s); }
        Ta[p][q] = va;
        Tb[p][q] = vb;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int e = tid + SYL_THREADS * k;
        Xs[e / SB][e % SB] = acc[k];
    }
    __syncthreads();
    for (int S = (br - 1) + (bc - 1); S >= 0; --S) {
        // solve the entries on diagonal p + q = S
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int e = tid + SYL_THREADS * k, p = e / SB, q = e % SB;
            if (p < br && q < bc && p + q == S) {
                cplx den = cadd(Ta[p][p], cconj(Tb[q][q]));
                Xs[p][q] = cdiv(Xs[p][q], den);
            }
        }
        __syncthreads();
        // eliminate them from the pending entries (p + q < S)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int e = tid + SYL_THREADS * k, p = e / SB, q = e % SB;
            if (p < br && q < bc && p + q < S) {
                cplx v = Xs[p][q];
                int r = S - q;                       // X[r][q] solved at this step, r > p
                if (r < br) {
                    cplx m = Ta[p][r], x = Xs[r][q];
                    v.x -= m.x * x.x - m.y * x.y;
                    v.y -= m.x * x.y + m.y * x.x;
                }
                r = S - p;                           // X[p][r] solved at this step, r > q
                if (r < bc) {
                    cplx x = Xs[p][r], m = Tb[q][r];
                    v.x -= x.x * m.x + x.y * m.y;
                    v.y -= x.y * m.x - x.x * m.y;
                }
                Xs[p][q] = v;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int e = tid + SYL_THREADS * k, p = e / SB, q = e % SB;
        if (p < br && q < bc) X[(long long)(r0 + p) * n + c0 + q] = Xs[p][q];
    }
}

}  // namespace

// Solves (T - s I) X + X (T - s I)^dag = C in place (X holds C on entry).
int trisylv_f64(const cplx* T, cplx* X, int n, cplx s, cudaStream_t st) {
    const int nb = (n + SB - 1) / SB;
    const size_t smem = 3 * SB * (SB + 1) * sizeof(cplx);
    if (lb_smem_attr((const void*)trisylv_f64_wave, (int)smem)) return -1;
    for (int w = 0; w <= 2 * nb - 2; ++w) {
        int lo = w - (nb - 1) > 0 ? w - (nb - 1) : 0;
        int hi = w < nb - 1 ? w : nb - 1;
        int cnt = hi - lo + 1;
        trisylv_f64_wave<<<cnt, SYL_THREADS, smem, st>>>(T, X, n, s, w, nb); lb_note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
