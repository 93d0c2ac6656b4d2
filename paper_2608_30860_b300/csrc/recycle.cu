// Right-preconditioned GMRES with Krylov subspace recycling (GCRO-DR; App. A.2: "after each cycle
// we retain a small harmonic-Ritz subspace (U, C) with L R U = C, passed to the next cycle and
// across successive solves"), and the three solvers built on it:
//   * steady_state_gmres : Alg. 3, L~_eta rho = eta I with P_0 = Precond(., 0, eta), warm start |0><0|;
//   * resolvent_solve    : (lam - L) X = B, lam > 0, preconditioned by R_lam^S (Sec. 3.1, 3.4);
//   * implicit_euler     : rho_{t+dt} = (1/dt) R_{1/dt}^L rho_t (Eq. resolvent, Sec. 4.3).
//
// The recycled method is that of Parks, de Sturler, Mackey, Johnson and Maiti (2006), written for
// the right-preconditioned operator B = A P, A = mu - L~_eta, P = Precond(., mu, eta) in Schur
// coordinates, where B = Id - K~ P (the right-preconditioning identity of Sec. 3.1): one Lyapunov
// solve and one jump term per step.  Each cycle with a recycled pair (U, C), B U = C, C orthonormal,
// runs m - k Arnoldi steps on (I - C C^H) B and minimises over range([U, V_{m-k}]); its k harmonic
// Ritz vectors of smallest |theta| become the next pair.  The small (m + 1) x m problems run in
// one-warp FP64 kernels; every operation on n x n operands runs in the library's kernels.
//
// Each solver is an FP64 residual-correction loop around the recycled GMRES: the residual of the
// full system is formed in FP64 in the original basis, moved to Schur coordinates, the correction
// is found by recycled GMRES (FP64 or tensor-core precision), mapped back and added.  In FP64 one
// GMRES cycle runs per correction, so the stopping test is evaluated after every cycle as Alg. 3
// prescribes; in mixed precision the correction runs to the low-precision floor first.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <vector>

#include "lb_internal.cuh"
#include "vecops.cuh"

namespace {

constexpr int LDS = KMAX + 2;        // leading dimension of the small column-major matrices
constexpr int RKMAX = 16;            // largest recycled subspace

// offsets (complex entries) of the small-matrix area h->gsm (column-major small matrices)
constexpr int OFF_G0 = 0;                              // G: rows x cols, ld LDS
constexpr int OFF_A = OFF_G0 + LDS * KMAX;             // Householder work, ld LDS
constexpr int OFF_F0 = OFF_A + LDS * KMAX;             // F: rows x cols, ld LDS
constexpr int OFF_F2 = OFF_F0 + LDS * KMAX;            // F S (transformed), ld LDS
constexpr int OFF_RHS = OFF_F2 + LDS * KMAX;
constexpr int OFF_RHS0 = OFF_RHS + LDS;
constexpr int OFF_Y = OFF_RHS0 + LDS;
constexpr int OFF_G = OFF_Y + LDS;
constexpr int OFF_GAM = OFF_G + LDS;                   // Gram matrix of [U^, V_p]: cols x cols, ld cols
constexpr int OFF_GEV = OFF_GAM + KMAX * KMAX;         // its eigenvalues
constexpr int OFF_GE = OFF_GEV + LDS;                  // its eigenvectors (Schur vectors), ld cols
constexpr int OFF_S = OFF_GE + KMAX * KMAX;            // S = E_r Lambda_r^{-1/2}: cols x r, ld cols
constexpr int OFF_M = OFF_S + KMAX * KMAX;             // M2: r x r, ld r
constexpr int OFF_EV = OFF_M + KMAX * KMAX;            // eigenvalues of M2
constexpr int OFF_EVEC = OFF_EV + LDS;                 // (eigenvectors of M2, unused)
constexpr int OFF_YS = OFF_EVEC + KMAX * KMAX;         // Schur vectors of M2: r x r, ld r
constexpr int OFF_Z = OFF_YS + KMAX * KMAX;            // Z = S Y_k: cols x knew, ld LDS
constexpr int OFF_GZ = OFF_Z + LDS * RKMAX;            // G Z, then Q_s: rows x knew, ld LDS
constexpr int OFF_ZR = OFF_GZ + LDS * RKMAX;           // Z R_s^{-1}: cols x knew, ld LDS
constexpr int OFF_BM = OFF_ZR + LDS * RKMAX;
constexpr int OFF_CU = OFF_BM + RKMAX * KMAX;
constexpr int OFF_UU = OFF_CU + RKMAX * RKMAX;
constexpr int OFF_VU = OFF_UU + RKMAX * RKMAX;
constexpr int OFF_C1 = OFF_VU + LDS * RKMAX;
constexpr int OFF_C2 = OFF_C1 + LDS;
constexpr int OFF_INV = OFF_C2 + LDS;
constexpr int GSM_ENTRIES = OFF_INV + 16;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Householder QR (one warp) of the rows x cols matrix A (ld LDS, in place: R on and above the
// diagonal), the reflectors applied to the ncb columns of Bm (ld LDS) and to the vector b (nullable);
// v: shared scratch of LDS entries
__device__ void warp_house_qr(cplx* A, int rows, int cols, cplx* Bm, int ncb, cplx* b, cplx* v) {
    const int lane = threadIdx.x;
    for (int c = 0; c < cols && c < rows; ++c) {
        double s2 = 0.0;
        for (int i = c + lane; i < rows; i += 32) s2 += cabs2(A[c * LDS + i]);
        s2 = wsum(s2);
        const cplx x0 = A[c * LDS + c];
        const double ax0 = hypot(x0.x, x0.y);
        const double nx = sqrt(s2);
        if (!(nx > 0.0)) continue;
        const cplx ph = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : cmake(1.0, 0.0);
        const cplx alpha = cscale(ph, -nx);
        const cplx v0 = csub(x0, alpha);
        const double vn2 = s2 - ax0 * ax0 + cabs2(v0);
        __syncwarp();
        for (int i = c + lane; i < rows; i += 32) v[i] = (i == c) ? v0 : A[c * LDS + i];
        __syncwarp();
        if (vn2 > 0.0) {
            const double f = 2.0 / vn2;
            for (int j = c + lane; j < cols + ncb; j += 32) {
                cplx* col = j < cols ? A + j * LDS : Bm + (j - cols) * LDS;
                cplx t = cmake(0, 0);
                for (int i = c; i < rows; ++i) cfma(t, cconj(v[i]), col[i]);
                t = cscale(t, f);
                for (int i = c; i < rows; ++i) col[i] = csub(col[i], cmul(t, v[i]));
            }
            if (b && lane == 0) {
                cplx t = cmake(0, 0);
                for (int i = c; i < rows; ++i) cfma(t, cconj(v[i]), b[i]);
                t = cscale(t, f);
                for (int i = c; i < rows; ++i) b[i] = csub(b[i], cmul(t, v[i]));
            }
        }
        __syncwarp();
    }
}

// X (cols x ncx, ld ldx) = R^{-1} Y (first cols rows of Y, ld LDS), R = upper(A[:cols, :cols]); lanes
// take columns; a zero pivot gives 0
__device__ void warp_back_subst(const cplx* A, int cols, const cplx* Y, int ncx, cplx* X, int ldx) {
    for (int j = threadIdx.x; j < ncx; j += 32) {
        for (int i = cols - 1; i >= 0; --i) {
            cplx acc = Y[j * LDS + i];
            for (int l = i + 1; l < cols; ++l) acc = csub(acc, cmul(A[l * LDS + i], X[j * ldx + l]));
            const cplx d = A[i * LDS + i];
            X[j * ldx + i] = (d.x == 0.0 && d.y == 0.0) ? cmake(0, 0) : cdiv(acc, d);
        }
    }
}

// One warp.  The augmented relation B [U^, V_p] = [C, V_{p+1}] G with G = [[D, Bm], [0, Hbar]]
// (rows = kk + p + 1, cols = kk + p; D = diag(dU)); the least-squares update y = argmin ||G y - beta e_kk||
// by Householder QR, g = beta e_kk - G y, res = ||g||; F = [C, V_{p+1}]^H [U^, V_p] = [[CU, 0], [VU, I]]
// and the Gram matrix Gamma = [U^, V_p]^H [U^, V_p] = [[UU, VU_p^H], [VU_p, I]] for the harmonic Ritz
// step.  Column-major, leading dimension LDS (Gamma: ld cols).
__global__ void k_gcro_small(int kk, int p, const double* __restrict__ dU, const cplx* __restrict__ Bm,
                             const cplx* __restrict__ Hb, int ldh, const cplx* __restrict__ CU,
                             const cplx* __restrict__ UU, const cplx* __restrict__ VU, double beta, cplx* gsm,
                             double* res) {
    cplx* G0 = gsm + OFF_G0;
    cplx* A = gsm + OFF_A;
    cplx* F = gsm + OFF_F0;
    cplx* rhs = gsm + OFF_RHS;
    cplx* rhs0 = gsm + OFF_RHS0;
    cplx* y = gsm + OFF_Y;
    cplx* g = gsm + OFF_G;
    cplx* Gam = gsm + OFF_GAM;
    __shared__ cplx v[LDS];
    const int lane = threadIdx.x;
    const int rows = kk + p + 1, cols = kk + p;
    for (int j = lane; j < cols; j += 32) {
        for (int i = 0; i < rows; ++i) {
            cplx gv = cmake(0, 0), fv = cmake(0, 0);
            if (j < kk) {
                if (i < kk) {
                    gv = cmake(i == j ? dU[j] : 0.0, 0.0);
                    fv = CU[j * RKMAX + i];
                } else {
                    fv = VU[j * LDS + (i - kk)];
                }
            } else {
                const int jj = j - kk;
                if (i < kk) {
                    gv = Bm[jj * RKMAX + i];
                } else {
                    const int ii = i - kk;
                    gv = (ii <= jj + 1) ? Hb[(long long)jj * ldh + ii] : cmake(0, 0);
                    fv = cmake(ii == jj ? 1.0 : 0.0, 0.0);
                }
            }
            G0[j * LDS + i] = gv;
            A[j * LDS + i] = gv;
            F[j * LDS + i] = fv;
        }
        for (int i = 0; i < cols; ++i) {
            cplx gm;
            if (i < kk && j < kk) gm = UU[j * RKMAX + i];
            else if (i >= kk && j < kk) gm = VU[j * LDS + (i - kk)];
            else if (i < kk && j >= kk) gm = cconj(VU[i * LDS + (j - kk)]);
            else gm = cmake(i == j ? 1.0 : 0.0, 0.0);
            Gam[j * cols + i] = gm;
        }
    }
    for (int i = lane; i < rows; i += 32) {
        const cplx r = cmake(i == kk ? beta : 0.0, 0.0);
        rhs[i] = r;
        rhs0[i] = r;
    }
    __syncwarp();
    warp_house_qr(A, rows, cols, nullptr, 0, rhs, v);
    if (lane == 0) {
        for (int i = cols - 1; i >= 0; --i) {
            cplx acc = rhs[i];
            for (int l = i + 1; l < cols; ++l) acc = csub(acc, cmul(A[l * LDS + i], y[l]));
            const cplx d = A[i * LDS + i];
            y[i] = (d.x == 0.0 && d.y == 0.0) ? cmake(0, 0) : cdiv(acc, d);
        }
    }
    __syncwarp();
    double r2 = 0.0;
    for (int i = lane; i < rows; i += 32) {
        cplx acc = rhs0[i];
        for (int j = 0; j < cols; ++j) acc = csub(acc, cmul(G0[j * LDS + i], y[j]));
        g[i] = acc;
        r2 += cabs2(acc);
    }
    r2 = wsum(r2);
    if (lane == 0) res[0] = sqrt(r2);
}

// One warp.  From the eigenpairs (Lambda, E) of Gamma: S = E_r Lambda_r^{-1/2} over the eigenvalues above
// 1e-10 of the largest, so that [U^, V_p] S is orthonormal; then the harmonic Ritz problem on that
// basis, (G S)^H (G S) w = theta (G S)^H (F S) w, as M2 = R^{-1} Q^H (F S) with G S = Q R (eigenvalues
// 1 / theta).  rdim[0] = r (as a double).
__global__ void k_gcro_harm(int kk, int p, cplx* gsm, double* rdim) {
    const cplx* G0 = gsm + OFF_G0;
    const cplx* F0 = gsm + OFF_F0;
    const cplx* lam = gsm + OFF_GEV;
    const cplx* E = gsm + OFF_GE;
    cplx* S = gsm + OFF_S;
    cplx* A = gsm + OFF_A;
    cplx* F2 = gsm + OFF_F2;
    cplx* M = gsm + OFF_M;
    __shared__ cplx v[LDS];
    __shared__ int idx[KMAX];
    __shared__ int rs;
    const int lane = threadIdx.x;
    const int rows = kk + p + 1, cols = kk + p;
    if (lane == 0) {
        double lmax = 0.0;
        for (int i = 0; i < cols; ++i) lmax = fmax(lmax, lam[i].x);
        int r = 0;
        for (int i = 0; i < cols; ++i)
            if (lam[i].x > 1e-10 * lmax) idx[r++] = i;
        rs = r;
        rdim[0] = (double)r;
    }
    __syncwarp();
    const int r = rs;
    for (int c = lane; c < r; c += 32) {
        const double f = 1.0 / sqrt(lam[idx[c]].x);
        for (int i = 0; i < cols; ++i) S[c * cols + i] = cscale(E[idx[c] * cols + i], f);
    }
    __syncwarp();
    for (int c = lane; c < r; c += 32) {
        for (int i = 0; i < rows; ++i) {
            cplx a = cmake(0, 0), b = cmake(0, 0);
            for (int j = 0; j < cols; ++j) {
                cfma(a, G0[j * LDS + i], S[c * cols + j]);
                cfma(b, F0[j * LDS + i], S[c * cols + j]);
            }
            A[c * LDS + i] = a;
            F2[c * LDS + i] = b;
        }
    }
    __syncwarp();
    warp_house_qr(A, rows, r, F2, r, nullptr, v);
    warp_back_subst(A, r, F2, r, M, r);
}

// One warp.  Z = S Y_k (Y: the first knew Schur vectors of M2, ld r), GZ = G Z, Householder QR
// GZ = Q_s R_s with Q_s formed explicitly (rows x knew, at OFF_GZ), ZR = Z R_s^{-1}; ok[0] = 1 when the
// pivots of R_s stay above 1e-6 of the largest (else the previous recycled pair is kept: ||R_s^{-1}||
// multiplies the relation error of the pair)
__global__ void k_gcro_zupdate(int kk, int p, int r, int knew, cplx* gsm, double* ok) {
    const cplx* G0 = gsm + OFF_G0;
    const cplx* S = gsm + OFF_S;
    const cplx* Y = gsm + OFF_YS;
    cplx* Z = gsm + OFF_Z;
    cplx* GZ = gsm + OFF_GZ;
    cplx* ZR = gsm + OFF_ZR;
    cplx* Q = gsm + OFF_F2;     // explicit Q_s (rows x knew)
    __shared__ cplx v[LDS];
    const int lane = threadIdx.x;
    const int rows = kk + p + 1, cols = kk + p;
    for (int t = lane; t < knew; t += 32) {
        for (int i = 0; i < cols; ++i) {
            cplx a = cmake(0, 0);
            for (int c = 0; c < r; ++c) cfma(a, S[c * cols + i], Y[t * r + c]);
            Z[t * LDS + i] = a;
        }
    }
    __syncwarp();
    for (int t = lane; t < knew; t += 32) {
        for (int i = 0; i < rows; ++i) {
            cplx a = cmake(0, 0);
            for (int j = 0; j < cols; ++j) cfma(a, G0[j * LDS + i], Z[t * LDS + j]);
            GZ[t * LDS + i] = a;
        }
        for (int i = 0; i < rows; ++i) Q[t * LDS + i] = cmake(i == t ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();
    // QR of GZ: keep the reflectors to form Q_s = H_0 ... H_{knew-1} [I; 0]
    cplx* Vh = gsm + OFF_A;     // reflector c in column c (ld LDS), its squared norm in Vh[c * LDS + LDS - 1]
    for (int c = 0; c < knew; ++c) {
        double s2 = 0.0;
        for (int i = c + lane; i < rows; i += 32) s2 += cabs2(GZ[c * LDS + i]);
        s2 = wsum(s2);
        const cplx x0 = GZ[c * LDS + c];
        const double ax0 = hypot(x0.x, x0.y), nx = sqrt(s2);
        const cplx ph = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : cmake(1.0, 0.0);
        const cplx alpha = cscale(ph, -nx);
        const cplx v0 = csub(x0, alpha);
        const double vn2 = nx > 0.0 ? s2 - ax0 * ax0 + cabs2(v0) : 0.0;
        __syncwarp();
        for (int i = c + lane; i < rows; i += 32) v[i] = (i == c) ? v0 : GZ[c * LDS + i];
        __syncwarp();
        for (int i = lane; i < LDS - 1; i += 32) Vh[c * LDS + i] = (i >= c && i < rows) ? v[i] : cmake(0, 0);
        if (lane == 0) Vh[c * LDS + LDS - 1] = cmake(vn2, 0.0);
        if (vn2 > 0.0) {
            const double f = 2.0 / vn2;
            for (int j = c + lane; j < knew; j += 32) {
                cplx t = cmake(0, 0);
                for (int i = c; i < rows; ++i) cfma(t, cconj(v[i]), GZ[j * LDS + i]);
                t = cscale(t, f);
                for (int i = c; i < rows; ++i) GZ[j * LDS + i] = csub(GZ[j * LDS + i], cmul(t, v[i]));
            }
        }
        __syncwarp();
    }
    for (int c = knew - 1; c >= 0; --c) {
        const double vn2 = Vh[c * LDS + LDS - 1].x;
        if (vn2 > 0.0) {
            const double f = 2.0 / vn2;
            for (int j = lane; j < knew; j += 32) {
                cplx t = cmake(0, 0);
                for (int i = c; i < rows; ++i) cfma(t, cconj(Vh[c * LDS + i]), Q[j * LDS + i]);
                t = cscale(t, f);
                for (int i = c; i < rows; ++i) Q[j * LDS + i] = csub(Q[j * LDS + i], cmul(t, Vh[c * LDS + i]));
            }
        }
        __syncwarp();
    }
    // ZR = Z R_s^{-1}: row i of ZR solves x R_s = z_i (lanes take rows)
    for (int i = lane; i < cols; i += 32) {
        for (int t = 0; t < knew; ++t) {
            cplx acc = Z[t * LDS + i];
            for (int l = 0; l < t; ++l) acc = csub(acc, cmul(ZR[l * LDS + i], GZ[t * LDS + l]));
            const cplx d = GZ[t * LDS + t];
            ZR[t * LDS + i] = (d.x == 0.0 && d.y == 0.0) ? cmake(0, 0) : cdiv(acc, d);
        }
    }
    if (lane == 0) {
        double dmax = 0.0, dmin = INFINITY;
        for (int t = 0; t < knew; ++t) {
            const double a = hypot(GZ[t * LDS + t].x, GZ[t * LDS + t].y);
            dmax = fmax(dmax, a);
            dmin = fmin(dmin, a);
        }
        ok[0] = (knew > 0 && dmin > 1e-6 * dmax && isfinite(dmin)) ? 1.0 : 0.0;
    }
}

// a[i] += b[i]
__global__ void k_add_small(cplx* a, const cplx* b, int k) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) a[i] = cadd(a[i], b[i]);
}
// c[i] = a[i] / d[i]
__global__ void k_div_small(cplx* c, const cplx* a, const double* d, int k) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = cscale(a[i], 1.0 / d[i]);
}
// inv = 1 / nrm[1] (complex scalar); dst (nullable) = 1 / nrm[1]
__global__ void k_inv_norm(const double* nrm, cplx* inv, double* dst) {
    if (threadIdx.x == 0) {
        const double v = nrm[1] > 0.0 ? 1.0 / nrm[1] : 0.0;
        inv[0] = cmake(v, 0.0);
        if (dst) dst[0] = v;
    }
}

// R_out = c1 * herm_or_not(R) + c0 * B + shift I, the max-norm of it to out[0] (host reads); helper
// of the stopping tests below: out = max_e | a R_e' + b B_e + diag |, R' = (R + R^dag)/2 if herm
__global__ void k_stop_combo(const cplx* __restrict__ R, const cplx* __restrict__ Bm, int n, int herm, cplx a, cplx b,
                             cplx diag, double* part) {
    __shared__ double red[8];
    const long long len = (long long)n * n;
    double m = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        cplx r = R[e];
        if (herm) {
            const cplx rt = R[(long long)j * n + i];
            r = cmake(0.5 * (r.x + rt.x), 0.5 * (r.y - rt.y));
        }
        cplx v = cmul(a, r);
        if (Bm) v = cadd(v, cmul(b, Bm[e]));
        if (i == j) v = cadd(v, diag);
        m = fmax(m, hypot(v.x, v.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
        part[blockIdx.x] = m;
    }
}
__global__ void k_max_final(const double* part, int nb, double* out) {
    double m = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) m = fmax(m, part[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[0] = m;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int read_doubles(cudaStream_t s, const double* d, double* h, int k) {
    if (cudaMemcpyAsync(h, d, k * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : -1;
}

}  // namespace

size_t recycle_bytes(int n, int rk) {
    const size_t nn = (size_t)n * n;
    return 4 * (size_t)rk * nn * sizeof(cplx) + 6 * 256 + 2 * RKMAX * sizeof(double) + GSM_ENTRIES * sizeof(cplx);
}

void recycle_layout(lb_handle_s* h, char*& base, int rk) {
    const size_t nn = (size_t)h->n * h->n;
    auto take = [&](size_t bytes) {
        char* p = base;
        if (base) base += (bytes + 255) & ~size_t(255);
        return p;
    };
    h->rk = rk;
    h->Urc = reinterpret_cast<cplx*>(take(rk * nn * sizeof(cplx)));
    h->Crc = reinterpret_cast<cplx*>(take(rk * nn * sizeof(cplx)));
    h->Unw = reinterpret_cast<cplx*>(take(rk * nn * sizeof(cplx)));
    h->Cnw = reinterpret_cast<cplx*>(take(rk * nn * sizeof(cplx)));
    h->dU = reinterpret_cast<double*>(take(2 * RKMAX * sizeof(double)));
    h->gsm = reinterpret_cast<cplx*>(take(GSM_ENTRIES * sizeof(cplx)));
}

void recycle_forget(lb_handle_s* h) {
    h->rc_have = 0;
    h->rc_prec = -1;
}

// Solves (mu - L~_eta) delta = b in Schur coordinates (B = A P, P = Precond(., mu, eta)) from delta = 0
// by GCRO-DR(m, k) with the handle's recycled pair (kept when it belongs to the same (mu, eta,
// precision)).  Stops when the residual norm <= atol, after max_cycles cycles, or when three cycles in
// a row each reduce it by less than 10 %.  Uses V / hm (basis), X[5] (r), X[6] (P v), X[7] (jump output).
int gcrodr_solve(lb_handle_s* h, cudaStream_t s, const cplx* b, cplx* delta, double mu, double eta, int m,
                 int kreq, int max_cycles, double atol, int precision, int* steps, double* final_res, int* cycles_out) {
    const long long nn = (long long)h->n * h->n;
    const int k = std::min(std::min(kreq, h->rk), std::max(0, m - 2));
    cplx* r = h->X[5];
    cplx* pv = h->X[6];
    cplx* gsm = h->gsm;
    double* res_d = h->dscal + 12;
    if (h->rc_prec != precision || h->rc_mu != mu || h->rc_eta != eta || k == 0) recycle_forget(h);
    const int k_lim = h->rc_have;
    h->rc_mu = mu;
    h->rc_eta = eta;
    h->rc_prec = precision;
    auto Bop = [&](const cplx* v, cplx* w) -> int {
        // B v = v - K~ P v  (right-preconditioning identity, Sec. 3.1)
        if (precond_apply(h, s, v, pv, mu, eta, precision, 0)) return -1;
        if (precision == LB_PREC_MIXED && h->mixed_ready) {
            if (jump_mixed(h, s, pv, w, -1.0)) return -1;
        } else if (jump_f64(h, s, h->Lt, pv, w, cmake(-1, 0), cmake(0, 0))) {
            return -1;
        }
        return vec_axpby(w, v, nn, cmake(1, 0), cmake(1, 0), s);
    };
    if (vec_scale_copy(delta, b, nn, cmake(0, 0), s)) return -1;
    if (vec_scale_copy(r, b, nn, cmake(1, 0), s)) return -1;
    int kk = std::min(k_lim, k);
    if (kk > 0) {
        // delta = P U C^H r, r -= C C^H r  (U scaled by 1/dU: B (u^_i / dU_i) = c_i)
        cplx* c1 = gsm + OFF_C1;
        cplx* c2 = gsm + OFF_C2;
        if (vec_dot_block(h->Crc, nn, kk, r, nn, c1, h->part, 0, s)) return -1;
        k_div_small<<<1, 32, 0, s>>>(c2, c1, h->dU, kk); lb_note_launch();
        if (vec_gemv(h->X[7], h->Urc, nn, kk, c2, nn, 1.0, 0, s)) return -1;
        if (precond_apply(h, s, h->X[7], pv, mu, eta, precision, 0)) return -1;
        if (vec_axpby(delta, pv, nn, cmake(1, 0), cmake(1, 0), s)) return -1;
        if (vec_gemv(r, h->Crc, nn, kk, c1, nn, -1.0, 1, s)) return -1;
    }
    if (vec_norms(r, nn, h->dpart, h->dscal, s)) return -1;
    double nr[2];
    if (read_doubles(s, h->dscal, nr, 2)) return -1;
    double beta = nr[1], prev = INFINITY;
    int cyc = 0, poor = 0;
    for (; cyc < max_cycles && beta > atol; ++cyc) {
        const int p = m - kk;
        if (vec_scale_copy(h->V, r, nn, cmake(1.0 / beta, 0), s)) return -1;
        cplx* Bm = gsm + OFF_BM;
        cplx* c1 = gsm + OFF_C1;
        int j = 0;
        OpFn op = [&](const cplx* v, cplx* w) -> int {
            if (Bop(v, w)) return -1;
            if (kk > 0) {
                // project out C twice; column j of Bm = C^H B v_j
                cplx* col = Bm + (size_t)j * RKMAX;
                if (vec_dot_block(h->Crc, nn, kk, w, nn, col, h->part, 0, s)) return -1;
                if (vec_gemv(w, h->Crc, nn, kk, col, nn, -1.0, 1, s)) return -1;
                if (vec_dot_block(h->Crc, nn, kk, w, nn, c1, h->part, 0, s)) return -1;
                if (vec_gemv(w, h->Crc, nn, kk, c1, nn, -1.0, 1, s)) return -1;
                k_add_small<<<1, 32, 0, s>>>(col, c1, kk); lb_note_launch();
            }
            ++j;
            return 0;
        };
        int pd = 0;
        if (arnoldi_cycle(h, s, h->V, h->hm, 0, p, op, &pd)) return -1;
        *steps += pd;
        // V[pd] (zero after a breakdown) completes V_{pd+1}
        cplx* CU = gsm + OFF_CU;
        cplx* UU = gsm + OFF_UU;
        cplx* VU = gsm + OFF_VU;
        for (int t = 0; t < kk; ++t) {
            if (vec_dot_block(h->Crc, nn, kk, h->Urc + t * nn, nn, CU + t * RKMAX, h->part, 0, s)) return -1;
            if (vec_dot_block(h->Urc, nn, kk, h->Urc + t * nn, nn, UU + t * RKMAX, h->part, 0, s)) return -1;
            if (vec_dot_block(h->V, nn, pd + 1, h->Urc + t * nn, nn, VU + t * LDS, h->part, 0, s)) return -1;
        }
        k_gcro_small<<<1, 32, 0, s>>>(kk, pd, h->dU, Bm, h->hm, h->ldh, CU, UU, VU, beta, gsm, res_d); lb_note_launch();
        const int cols = kk + pd;
        const cplx* y = gsm + OFF_Y;
        const cplx* g = gsm + OFF_G;
        // delta += P (U^ y_U + V_p y_V)
        cplx* tmp = h->X[7];
        if (kk > 0) {
            if (vec_gemv(tmp, h->Urc, nn, kk, y, nn, 1.0, 0, s)) return -1;
            if (vec_gemv(tmp, h->V, nn, pd, y + kk, nn, 1.0, 1, s)) return -1;
        } else if (vec_gemv(tmp, h->V, nn, pd, y, nn, 1.0, 0, s)) {
            return -1;
        }
        if (precond_apply(h, s, tmp, pv, mu, eta, precision, 0)) return -1;
        if (vec_axpby(delta, pv, nn, cmake(1, 0), cmake(1, 0), s)) return -1;
        // r = C g_C + V_{p+1} g_V
        if (kk > 0) {
            if (vec_gemv(r, h->Crc, nn, kk, g, nn, 1.0, 0, s)) return -1;
            if (vec_gemv(r, h->V, nn, pd + 1, g + kk, nn, 1.0, 1, s)) return -1;
        } else if (vec_gemv(r, h->V, nn, pd + 1, g, nn, 1.0, 0, s)) {
            return -1;
        }
        // new recycled pair: harmonic Ritz vectors of smallest |theta| on an orthonormal basis of
        // range([U^, V_p]) (its Gram matrix's well-conditioned eigenvectors: once a cycle has nearly
        // converged, [U^, V_p] is numerically rank-deficient and its null directions would pass for
        // spurious harmonic Ritz vectors), as Schur vectors of the selected values; C = [C, V] Q_s and
        // U = [U^, V_p] Z R_s^{-1} from the small QR G Z = Q_s R_s, so B U = C holds by construction
        if (k > 0 && cols > 0) {
            if (small_schur(gsm + OFF_GAM, cols, cols, 0, 0, 0, gsm + OFF_GEV, gsm + OFF_EVEC, nullptr, gsm + OFF_GE,
                            h->dinfo, s))
                return -1;
            k_gcro_harm<<<1, 32, 0, s>>>(kk, pd, gsm, h->dscal + 13); lb_note_launch();
            double rd[2];
            if (read_doubles(s, h->dscal + 12, rd, 2)) return -1;
            const int rdim = (int)rd[1];
            const int knew = std::min(k, rdim);
            double ok = 0.0;
            // a cycle that met the tolerance leaves the pair as it was: the end of a converged Krylov space
            // is rounding noise, and every update carries the previous pair's relation error forward
            // multiplied by ||R_s^{-1}||, so updating from such cycles lets B U = C drift over a sequence of
            // solves (shift-invert applications) until the estimated residuals no longer mean anything
            if (knew > 0 && rd[0] > atol) {
                if (small_schur(gsm + OFF_M, rdim, rdim, 0, 1, knew, gsm + OFF_EV, gsm + OFF_EVEC, nullptr,
                                gsm + OFF_YS, h->dinfo, s))
                    return -1;
                k_gcro_zupdate<<<1, 32, 0, s>>>(kk, pd, rdim, knew, gsm, h->dscal + 15); lb_note_launch();
                if (read_doubles(s, h->dscal + 15, &ok, 1)) return -1;
            }
            if (ok > 0.5) {
                const cplx* QS = gsm + OFF_F2;
                const cplx* ZR = gsm + OFF_ZR;
                cplx* inv = gsm + OFF_INV;
                double* dnew = h->dU + RKMAX;
                for (int t = 0; t < knew; ++t) {
                    cplx* ut = h->Unw + t * nn;
                    cplx* ct = h->Cnw + t * nn;
                    const cplx* qt = QS + (size_t)t * LDS;
                    const cplx* zt = ZR + (size_t)t * LDS;
                    if (kk > 0) {
                        if (vec_gemv(ct, h->Crc, nn, kk, qt, nn, 1.0, 0, s)) return -1;
                        if (vec_gemv(ct, h->V, nn, pd + 1, qt + kk, nn, 1.0, 1, s)) return -1;
                        if (vec_gemv(ut, h->Urc, nn, kk, zt, nn, 1.0, 0, s)) return -1;
                        if (vec_gemv(ut, h->V, nn, pd, zt + kk, nn, 1.0, 1, s)) return -1;
                    } else {
                        if (vec_gemv(ct, h->V, nn, pd + 1, qt, nn, 1.0, 0, s)) return -1;
                        if (vec_gemv(ut, h->V, nn, pd, zt, nn, 1.0, 0, s)) return -1;
                    }
                    // unit columns for U: u^_t = u_t / ||u_t||, B u^_t = dU_t c_t
                    if (vec_norms(ut, nn, h->dpart, h->dscal + 2, s)) return -1;
                    k_inv_norm<<<1, 32, 0, s>>>(h->dscal + 2, inv, dnew + t); lb_note_launch();
                    if (vec_scale_dev(ut, nn, inv, s)) return -1;
                }
                std::swap(h->Urc, h->Unw);
                std::swap(h->Crc, h->Cnw);
                if (cudaMemcpyAsync(h->dU, dnew, knew * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    return -1;
                h->rc_have = knew;
                kk = knew;
            }
        }
        double rr = 0.0;
        if (read_doubles(s, res_d, &rr, 1)) return -1;
        prev = beta;
        beta = rr;
        // stagnation: three cycles in a row that gain less than 10 % (a recycled solve often stalls
        // for a cycle or two until the pair has captured the slow direction, then resumes)
        poor = beta > 0.9 * prev ? poor + 1 : 0;
        if (poor >= 3) { ++cyc; break; }
    }
    *final_res = beta;
    if (cycles_out) *cycles_out += cyc;
    return 0;
}

// ============================================================================ refined shifted solve
// Stop test of the shifted solves, given x (original basis) and R = b - (mu - L~_eta)(x) (FP64,
// original basis): returns 1 when done, writing the tested quantity to *val.
typedef std::function<int(const cplx* x, const cplx* R, double* val)> StopFn;

// x (original basis, in/out: warm start) solves (mu - L~_eta) x = b by FP64 residual correction
// around recycled GMRES.  Returns LB_OK on stop, LB_NOT_CONVERGED (x is the last iterate) otherwise.
static lb_status shifted_solve(lb_handle_s* h, cudaStream_t s, double mu, double eta, const cplx* b, cplx* x,
                               const lb_opts& o, const StopFn& stop, int max_outer, lb_info* inf) {
    const int n = h->n;
    const long long nn = (long long)n * n;
    cplx* R = h->X[1];
    cplx* rt = h->X[2];
    cplx* dt = h->X[3];
    cplx* tmp = h->X[4];
    const int prec = o.precision;
    const int m = std::min(o.gmres_m, h->vcap - 1);
    double prev = INFINITY;
    for (int it = 0; it <= max_outer; ++it) {
        // R = b - mu x + L(x) + eta Tr(x) I
        if (lindbladian_f64(h, s, x, R)) return LB_CUDA_ERROR;
        if (vec_axpby(R, x, nn, cmake(-mu, 0), cmake(1, 0), s)) return LB_CUDA_ERROR;
        if (vec_axpby(R, b, nn, cmake(1, 0), cmake(1, 0), s)) return LB_CUDA_ERROR;
        if (eta != 0.0) {
            if (mat_trace(x, n, h->scal + 11, s)) return LB_CUDA_ERROR;
            if (mat_add_diag_dev(R, n, h->scal + 11, eta, s)) return LB_CUDA_ERROR;
        }
        double val = INFINITY;
        const int done = stop(x, R, &val);
        if (done < 0) return LB_CUDA_ERROR;
        inf->residual_max = val;
        if (done) return LB_OK;
        if (it == max_outer) break;
        // mixed precision: a correction that no longer lowers the tested quantity has hit the floor
        if (prec == LB_PREC_MIXED && !(val < 0.5 * prev) && it > 1) break;
        prev = std::min(prev, val);
        if (change_basis(h, s, R, rt, tmp, 1)) return LB_CUDA_ERROR;
        if (vec_norms(rt, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
        double nr[2];
        if (read_doubles(s, h->dscal, nr, 2)) return LB_CUDA_ERROR;
        int steps = 0, cycles = 0;
        double res = 0.0;
        // FP64: one cycle per correction, so that the test above runs after every cycle (Alg. 3);
        // mixed: cycles until the tensor-core floor (~1e-6 relative) or stagnation
        const int cyc = prec == LB_PREC_MIXED ? 6 : 1;
        const double atol = prec == LB_PREC_MIXED ? 1e-6 * nr[1] : 1e-15 * nr[1];
        if (gcrodr_solve(h, s, rt, dt, mu, eta, m, o.recycle_k, cyc, atol, prec, &steps, &res, &cycles))
            return LB_CUDA_ERROR;
        inf->gmres_steps += steps;
        inf->phi_applies += steps;
        inf->restarts += cycles;
        inf->refine_steps += 1;
        if (change_basis(h, s, dt, tmp, R, 0)) return LB_CUDA_ERROR;
        if (vec_axpby(x, tmp, nn, cmake(1, 0), cmake(1, 0), s)) return LB_CUDA_ERROR;
    }
    return LB_NOT_CONVERGED;
}

// max-norm of a R' + c B + diag I (R' = hermitised R if herm), on the device, read back
static int stop_norm(lb_handle_s* h, cudaStream_t s, const cplx* R, const cplx* Bm, int herm, cplx a, cplx c,
                     cplx diag, double* out) {
    constexpr int NB = 592;
    k_stop_combo<<<NB, 256, 0, s>>>(R, Bm, h->n, herm, a, c, diag, h->dpart); lb_note_launch();
    k_max_final<<<1, 32, 0, s>>>(h->dpart, NB, h->dscal + 14); lb_note_launch();
    return read_doubles(s, h->dscal + 14, out, 1);
}

static int read_trace(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* out) {
    if (mat_trace(X, h->n, h->scal + 12, s)) return -1;
    if (cudaMemcpyAsync(out, h->scal + 12, sizeof(cplx), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : -1;
}

// (lam - L) X = B with lam > 0 (eta = 0): stop when ||(lam - L)(X^) - B||_max < tol, X^ the iterate
// hermitised (B Hermitian) and rescaled to its exact trace Tr B / lam (Sec. 3.4).  On return X = X^.
static lb_status resolvent_core(lb_handle_s* h, cudaStream_t s, double lam, const cplx* B, cplx* X, double tol,
                                int herm, const lb_opts& o, int max_outer, lb_info* inf) {
    const int n = h->n;
    const long long nn = (long long)n * n;
    cplx trB;
    if (read_trace(h, s, B, &trB)) return LB_CUDA_ERROR;
    const std::complex<double> target = std::complex<double>(trB.x, trB.y) / lam;
    std::complex<double> cfin(1.0, 0.0);
    StopFn stop = [&](const cplx* x, const cplx* R, double* val) -> int {
        cplx trx;
        if (read_trace(h, s, x, &trx)) return -1;
        std::complex<double> t(trx.x, herm ? 0.0 : trx.y);
        const std::complex<double> c = std::abs(t) > 0.0 ? target / t : std::complex<double>(1.0, 0.0);
        // (lam - L)(c x') - B = c (B' - R') - B, primes = hermitised (B' = B for Hermitian B)
        if (stop_norm(h, s, R, B, herm, cmake(-c.real(), -c.imag()), cmake(c.real() - 1.0, c.imag()), cmake(0, 0),
                      val))
            return -1;
        cfin = c;
        return *val < tol ? 1 : 0;
    };
    lb_status st = shifted_solve(h, s, lam, 0.0, B, X, o, stop, max_outer, inf);
    if (st < 0) return st;
    if (herm && mat_hermitize(X, X, n, s)) return LB_CUDA_ERROR;
    if (vec_scale_copy(X, X, nn, cmake(cfin.real(), cfin.imag()), s)) return LB_CUDA_ERROR;
    return st;
}

static int is_hermitian(lb_handle_s* h, cudaStream_t s, const cplx* B) {
    double v = 0.0;
    // max |B - B^dag| / 2 = max |hermitised(B) - B|
    if (stop_norm(h, s, B, B, 1, cmake(1, 0), cmake(-1, 0), cmake(0, 0), &v)) return -1;
    return v == 0.0 ? 1 : 0;
}

// every entry finite (the sum of squares is finite exactly when no entry is NaN or Inf and none is
// above ~1e154)
static bool all_finite(lb_handle_s* h, cudaStream_t s, const cplx* X, long long len) {
    if (vec_norms(X, len, h->dpart, h->dscal, s)) return false;
    double v[2];
    if (read_doubles(s, h->dscal, v, 2)) return false;
    return std::isfinite(v[1]);
}

static lb_status begin_solve(lb_handle_s* h, const lb_opts* opts, lb_opts& o) {
    o = h->opts;
    if (opts) o = *opts;
    if (o.gmres_m < 4 || o.gmres_m + 1 > h->vcap || o.gmres_m > KMAX || o.recycle_k < 0) return LB_INVALID_ARG;
    if (o.precision == LB_PREC_MIXED && !h->mixed_ready) return LB_NOT_IMPLEMENTED;
    return LB_OK;
}

static void fill_common(lb_handle_s* h, lb_info& inf) {
    inf.schur_backward_err = h->schur_err;
    inf.min_abs_re_T = h->min_re_T;
    inf.setup_ms = h->setup_ms;
    inf.cond_eig = h->cond_eig;
    inf.route = h->eig_active ? LB_ROUTE_EIG : LB_ROUTE_SCHUR;
}

// ============================================================================ C ABI
extern "C" {

static lb_status steady_state_gmres_body(lindblad_handle h, void* rho_dev, const lb_opts* opts, lb_info* info, void* stream) {
    if (!h || !rho_dev) return LB_INVALID_ARG;
    lb_opts o;
    lb_status st = begin_solve(h, opts, o);
    if (st != LB_OK) return st;
    if (h->case1) return LB_S_SINGULAR;
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = now_ms();
    const int n = h->n;
    const long long nn = (long long)n * n;
    lb_info inf{};
    fill_common(h, inf);
    st = precond_prepare(h, s, 0.0, o.eta, o.precision, 0);
    if (st != LB_OK) return st;
    cplx* x = (cplx*)rho_dev;
    cplx* b = h->bk0;
    // L~_eta rho = eta I  <=>  (0 - L~_eta) rho = -eta I ; warm start |0><0|
    if (mat_eye(b, n, cmake(-o.eta, 0), s)) return LB_CUDA_ERROR;
    if (vec_scale_copy(x, x, nn, cmake(0, 0), s)) return LB_CUDA_ERROR;
    const cplx one = cmake(1, 0);
    if (cudaMemcpyAsync(x, &one, sizeof(cplx), cudaMemcpyHostToDevice, s) != cudaSuccess) return LB_CUDA_ERROR;
    double best = INFINITY;
    double rfro_best = 0.0;
    // the test of Alg. 3 on rho^ = herm(x) / Re Tr x: L(rho^) = (herm(R) - eta (Re Tr x - 1) I) / Re Tr x
    StopFn stop = [&](const cplx* xx, const cplx* R, double* val) -> int {
        cplx trx;
        if (read_trace(h, s, xx, &trx)) return -1;
        const double t = trx.x;
        if (!(std::fabs(t) > 0.0)) { *val = INFINITY; return 0; }
        if (stop_norm(h, s, R, nullptr, 1, cmake(1.0 / t, 0), cmake(0, 0), cmake(-o.eta * (t - 1.0) / t, 0), val))
            return -1;
        if (*val < best) {
            best = *val;
            if (cudaMemcpyAsync(h->best, xx, nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s) != cudaSuccess) return -1;
        }
        return *val < o.tol ? 1 : 0;
    };
    const int max_outer = o.precision == LB_PREC_MIXED ? o.max_refine + 4 : o.max_restarts;
    st = shifted_solve(h, s, 0.0, o.eta, b, x, o, stop, max_outer, &inf);
    if (st < 0) return st;
    // return the best iterate, hermitised and trace-normalised, with its residual recomputed
    if (hermitize_normalize(h, s, h->best, x, h->X[4])) return LB_CUDA_ERROR;
    double rmax = 0.0;
    if (residual_norms(h, s, x, h->X[1], &rmax, &rfro_best)) return LB_CUDA_ERROR;
    inf.residual_max = rmax;
    inf.residual_fro = rfro_best;
    st = rmax < o.tol ? LB_OK : LB_NOT_CONVERGED;
    inf.status = st;
    inf.solve_ms = now_ms() - t0;
    if (info) *info = inf;
    return st;
}

lb_status steady_state_gmres(lindblad_handle h, void* rho_dev, const lb_opts* opts, lb_info* info, void* stream) {
    return device_error_guard(h, (cudaStream_t)stream, steady_state_gmres_body(h, rho_dev, opts, info, stream));
}

static lb_status resolvent_solve_body(lindblad_handle h, double lam, const void* B_dev, void* X_dev, const lb_opts* opts,
                          lb_info* info, void* stream) {
    if (!h || !B_dev || !X_dev || B_dev == X_dev || !(lam > 0.0) || !std::isfinite(lam)) return LB_INVALID_ARG;
    lb_opts o;
    lb_status st = begin_solve(h, opts, o);
    if (st != LB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = now_ms();
    const long long nn = (long long)h->n * h->n;
    lb_info inf{};
    fill_common(h, inf);
    const cplx* B = (const cplx*)B_dev;
    cplx* X = (cplx*)X_dev;
    if (!all_finite(h, s, B, nn)) return LB_INVALID_ARG;
    const int herm = is_hermitian(h, s, B);
    if (herm < 0) return LB_CUDA_ERROR;
    if (vec_scale_copy(X, B, nn, cmake(0, 0), s)) return LB_CUDA_ERROR;
    const int max_outer = o.precision == LB_PREC_MIXED ? o.max_refine + 4 : o.max_restarts;
    st = resolvent_core(h, s, lam, B, X, o.tol, herm, o, max_outer, &inf);
    if (st < 0) return st;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LB_CUDA_ERROR;
    inf.status = st;
    inf.solve_ms = now_ms() - t0;
    if (info) *info = inf;
    return st;
}

lb_status resolvent_solve(lindblad_handle h, double lam, const void* B_dev, void* X_dev, const lb_opts* opts,
                          lb_info* info, void* stream) {
    return device_error_guard(h, (cudaStream_t)stream, resolvent_solve_body(h, lam, B_dev, X_dev, opts, info, stream));
}

static lb_status implicit_euler_body(lindblad_handle h, const void* rho0_dev, double dt, int nsteps, void* rho_dev,
                         void* traj_dev, const lb_opts* opts, lb_info* info, void* stream) {
    if (!h || !rho0_dev || !rho_dev || rho0_dev == rho_dev || !(dt > 0.0) || !std::isfinite(dt) || nsteps < 1)
        return LB_INVALID_ARG;
    lb_opts o;
    lb_status st = begin_solve(h, opts, o);
    if (st != LB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = now_ms();
    const long long nn = (long long)h->n * h->n;
    const size_t bytes = (size_t)nn * sizeof(cplx);
    const double lam = 1.0 / dt;
    lb_info inf{};
    fill_common(h, inf);
    cplx* rho = (cplx*)rho_dev;
    cplx* b = h->bk0;
    if (cudaMemcpyAsync(rho, rho0_dev, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return LB_CUDA_ERROR;
    if (!all_finite(h, s, rho, nn)) return LB_INVALID_ARG;
    const int herm = is_hermitian(h, s, rho);
    if (herm < 0) return LB_CUDA_ERROR;
    double worst = 0.0;
    lb_status agg = LB_OK;
    for (int k = 0; k < nsteps; ++k) {
        // (1/dt - L) rho_{k+1} = rho_k / dt, warm start rho_k, tolerance relative to ||rho_k / dt||_max
        if (vec_scale_copy(b, rho, nn, cmake(lam, 0), s)) return LB_CUDA_ERROR;
        if (vec_norms(b, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
        double bn[2];
        if (read_doubles(s, h->dscal, bn, 2)) return LB_CUDA_ERROR;
        lb_info si{};
        const int max_outer = o.precision == LB_PREC_MIXED ? o.max_refine + 4 : o.max_restarts;
        st = resolvent_core(h, s, lam, b, rho, o.tol * bn[0], herm, o, max_outer, &si);
        if (st < 0) return st;
        if (st != LB_OK) agg = st;
        worst = std::max(worst, si.residual_max / std::max(bn[0], 1e-300));
        inf.gmres_steps += si.gmres_steps;
        inf.phi_applies += si.phi_applies;
        inf.refine_steps += si.refine_steps;
        inf.restarts += si.restarts;
        if (traj_dev && cudaMemcpyAsync((cplx*)traj_dev + (size_t)k * nn, rho, bytes, cudaMemcpyDeviceToDevice, s) !=
                            cudaSuccess)
            return LB_CUDA_ERROR;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return LB_CUDA_ERROR;
    inf.residual_max = worst;
    inf.status = agg;
    inf.solve_ms = now_ms() - t0;
    if (info) *info = inf;
    return agg;
}

lb_status implicit_euler(lindblad_handle h, const void* rho0_dev, double dt, int nsteps, void* rho_dev,
                         void* traj_dev, const lb_opts* opts, lb_info* info, void* stream) {
    return device_error_guard(h, (cudaStream_t)stream, implicit_euler_body(h, rho0_dev, dt, nsteps, rho_dev, traj_dev, opts, info, stream));
}

}  // extern "C"
