// Small dense eigenproblems of the Krylov loops (m <= 64, FP64) as a warp-level device routine:
// Householder reduction to Hessenberg form (general input), implicitly shifted single-shift QR to
// complex Schur form (Wilkinson shift, exceptional shifts after 10 and 20 stalled sweeps),
// optional reordering of the Schur form by adjacent swaps (the Givens rotation that maps the 2 x 2
// block's second eigenvector onto e1), eigenvectors of the triangular factor by back substitution
// mapped back with Z and normalised.  Used by hess.cu (one warp per launch) and batched.cu (one
// warp per instance).  The QR sweep count is capped at 30 m; info = 1 reports a stall.
#pragma once
#include "common.cuh"


static __device__ __forceinline__ double cabsd(cplx a) { return hypot(a.x, a.y); }

static __device__ __forceinline__ cplx csqrt_d(cplx z) {
    double r = cabsd(z);
    if (r == 0.0) return cmake(0.0, 0.0);
    double t = sqrt(0.5 * (r + fabs(z.x)));
    if (z.x >= 0.0) return cmake(t, z.y / (2.0 * t));
    return cmake(fabs(z.y) / (2.0 * t), z.y >= 0.0 ? t : -t);
}

// c real, s complex with [c s; -conj(s) c] [x; y] = [r; 0]
static __device__ __forceinline__ void givens(cplx x, cplx y, double& c, cplx& s) {
    double ax = cabsd(x), ay = cabsd(y);
    if (ay == 0.0) { c = 1.0; s = cmake(0.0, 0.0); return; }
    if (ax == 0.0) { c = 0.0; s = cscale(cconj(y), 1.0 / ay); return; }
    double r = hypot(ax, ay);
    c = ax / r;
    s = cscale(cmul(cscale(x, 1.0 / ax), cconj(y)), 1.0 / r);
}

// rows k, k+1 of A (columns j0..m-1) <- G [row k; row k+1]
static __device__ __forceinline__ void rot_rows(cplx* A, int m, int ld, int k, int j0, double c, cplx s, int lane) {
    for (int j = j0 + lane; j < m; j += 32) {
        cplx a = A[k * ld + j], b = A[(k + 1) * ld + j];
        A[k * ld + j] = cadd(cscale(a, c), cmul(s, b));
        A[(k + 1) * ld + j] = csub(cscale(b, c), cmul(cconj(s), a));
    }
}
// columns k, k+1 of A (rows 0..imax) <- [col k, col k+1] G^dag
static __device__ __forceinline__ void rot_cols(cplx* A, int ld, int k, int imax, double c, cplx s, int lane) {
    for (int i = lane; i <= imax; i += 32) {
        cplx a = A[i * ld + k], b = A[i * ld + k + 1];
        A[i * ld + k] = cadd(cscale(a, c), cmul(b, cconj(s)));
        A[i * ld + k + 1] = csub(cscale(b, c), cmul(a, s));
    }
}

static __device__ __forceinline__ double order_key(cplx v, int order) {
    if (order == 1) return cabsd(v);                                   // largest |nu| first
    return -cabsd(csub(v, cmake(1.0, 0.0))) + 1e-300 * v.x;            // nearest 1 first
}

// One warp (lane = threadIdx.x & 31) computes the ordered Schur form / eigenpairs; A, Z, Vt are
// m x (m + 1) shared-memory buffers, hv (>= m entries), rot_s, rot_c shared scratch.
static __device__ void small_schur_warp(const cplx* __restrict__ Ain, int lda, int m, int hess_in, int order, int nsel,
                                 cplx* __restrict__ evals, cplx* __restrict__ evecs, cplx* __restrict__ Tout,
                                 cplx* __restrict__ Zout, int* info, cplx* A, cplx* Z, cplx* Vt, cplx* hv,
                                 cplx& rot_s, double& rot_c) {
    const int lane = threadIdx.x & 31;
    const int ld = m + 1;   // padded row stride: column sweeps hit distinct banks
    const double eps = 2.220446049250313e-16;

    for (int e = lane; e < m * m; e += 32) {
        int i = e / m, j = e % m;
        cplx a = Ain[(long long)j * lda + i];             // column-major input
        if (hess_in && i > j + 1) a = cmake(0.0, 0.0);
        A[i * ld + j] = a;
        Z[i * ld + j] = cmake(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();

    // 1. Householder reduction to Hessenberg form
    if (!hess_in) {
        for (int k = 0; k + 2 < m; ++k) {
            double nrm2 = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) nrm2 += cabs2(A[i * ld + k]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
            double xn = sqrt(nrm2);
            cplx x0 = A[(k + 1) * ld + k];
            double sub = xn * xn - cabs2(x0);
            if (xn == 0.0 || sub <= 1e-300 * xn * xn) continue;      // already zero below subdiagonal
            double ax0 = cabsd(x0);
            cplx ph = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : cmake(1.0, 0.0);
            cplx alpha = cscale(ph, -xn);
            // v = x - alpha e1, normalised
            for (int i = k + 1 + lane; i < m; i += 32) hv[i] = A[i * ld + k];
            __syncwarp();
            if (lane == 0) hv[k + 1] = csub(hv[k + 1], alpha);
            __syncwarp();
            double vn = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) vn += cabs2(hv[i]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vn += __shfl_xor_sync(0xffffffffu, vn, o);
            double inv = 1.0 / sqrt(vn);
            for (int i = k + 1 + lane; i < m; i += 32) hv[i] = cscale(hv[i], inv);
            __syncwarp();
            // A <- (I - 2 v v^H) A
            for (int j = k + lane; j < m; j += 32) {
                cplx sacc = cmake(0.0, 0.0);
                for (int i = k + 1; i < m; ++i) cfma(sacc, cconj(hv[i]), A[i * ld + j]);
                for (int i = k + 1; i < m; ++i) A[i * ld + j] = csub(A[i * ld + j], cscale(cmul(hv[i], sacc), 2.0));
            }
            __syncwarp();
            // A <- A (I - 2 v v^H) ; Z <- Z (I - 2 v v^H)
            for (int i = lane; i < m; i += 32) {
                cplx sa = cmake(0.0, 0.0), sz = cmake(0.0, 0.0);
                for (int j = k + 1; j < m; ++j) { cfma(sa, A[i * ld + j], hv[j]); cfma(sz, Z[i * ld + j], hv[j]); }
                for (int j = k + 1; j < m; ++j) {
                    A[i * ld + j] = csub(A[i * ld + j], cscale(cmul(sa, cconj(hv[j])), 2.0));
                    Z[i * ld + j] = csub(Z[i * ld + j], cscale(cmul(sz, cconj(hv[j])), 2.0));
                }
            }
            __syncwarp();
            for (int i = k + 2 + lane; i < m; i += 32) A[i * ld + k] = cmake(0.0, 0.0);
            __syncwarp();
        }
    }

    // 2. shifted QR to complex Schur form
    int hi = m - 1, iter = 0, total = 0, stalled = 0;
    const int max_total = 30 * m;
    while (hi > 0) {
        if (total >= max_total) { stalled = 1; break; }
        int l = hi;
        while (l > 0) {
            double sub = cabsd(A[l * ld + l - 1]);
            double dg = cabsd(A[l * ld + l]) + cabsd(A[(l - 1) * ld + l - 1]);
            if (sub <= eps * dg || sub < 1e-300) break;
            --l;
        }
        __syncwarp();
        if (l > 0 && lane == 0) A[l * ld + l - 1] = cmake(0.0, 0.0);
        __syncwarp();
        if (l == hi) { --hi; iter = 0; continue; }
        cplx mu;
        cplx d = A[hi * ld + hi];
        if (iter == 10 || iter == 20) {
            double s = fabs(A[hi * ld + hi - 1].x) + fabs(A[hi * ld + hi - 1].y);
            mu = cadd(d, cmake(0.75 * s, 0.0));
        } else {
            cplx a = A[(hi - 1) * ld + hi - 1], b = A[(hi - 1) * ld + hi], c = A[hi * ld + hi - 1];
            cplx half = cscale(csub(a, d), 0.5);
            cplx disc = csqrt_d(cadd(cmul(half, half), cmul(b, c)));
            cplx mid = cscale(cadd(a, d), 0.5);
            cplx m1 = cadd(mid, disc), m2 = csub(mid, disc);
            mu = (cabs2(csub(m1, d)) <= cabs2(csub(m2, d))) ? m1 : m2;
        }
        for (int k = l; k < hi; ++k) {
            if (lane == 0) {
                cplx x, y;
                if (k == l) { x = csub(A[l * ld + l], mu); y = A[(l + 1) * ld + l]; }
                else { x = A[k * ld + k - 1]; y = A[(k + 1) * ld + k - 1]; }
                double c; cplx s;
                givens(x, y, c, s);
                rot_c = c;
                rot_s = s;
            }
            __syncwarp();
            const double c = rot_c;
            const cplx s = rot_s;
            rot_rows(A, m, ld, k, k == l ? l : k - 1, c, s, lane);
            __syncwarp();
            rot_cols(A, ld, k, min(k + 2, hi), c, s, lane);
            rot_cols(Z, ld, k, m - 1, c, s, lane);
            __syncwarp();
            if (k > l && lane == 0) A[(k + 1) * ld + k - 1] = cmake(0.0, 0.0);
            __syncwarp();
        }
        ++iter;
        ++total;
    }
    __syncwarp();

    // 3. reorder: the nsel best eigenvalues (by key) to the leading positions
    if (order != 0) {
        for (int pos = 0; pos < nsel && pos < m; ++pos) {
            int bi = pos;
            double bk = order_key(A[pos * ld + pos], order);
            for (int i = pos + 1; i < m; ++i) {
                double ki = order_key(A[i * ld + i], order);
                if (ki > bk + 1e-14 * fabs(bk)) { bk = ki; bi = i; }
            }
            for (int k = bi - 1; k >= pos; --k) {
                if (lane == 0) {
                    cplx t11 = A[k * ld + k], t22 = A[(k + 1) * ld + k + 1];
                    double c; cplx s;
                    givens(A[k * ld + k + 1], csub(t22, t11), c, s);
                    rot_c = c;
                    rot_s = s;
                }
                __syncwarp();
                const double c = rot_c;
                const cplx s = rot_s;
                rot_rows(A, m, ld, k, k, c, s, lane);
                __syncwarp();
                rot_cols(A, ld, k, k + 1, c, s, lane);
                rot_cols(Z, ld, k, m - 1, c, s, lane);
                __syncwarp();
                if (lane == 0) A[(k + 1) * ld + k] = cmake(0.0, 0.0);
                __syncwarp();
            }
        }
    }

    // 4. eigenvectors of the triangular factor, then y_p = Z v_p (skipped when evecs is null)
    for (int p = lane; p < m; p += 32) evals[p] = A[p * ld + p];
    if (evecs) {
        double tnorm = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) tnorm = fmax(tnorm, cabsd(A[i * ld + j]));
        const double small = fmax(eps * tnorm, 1e-300);
        for (int p = lane; p < m; p += 32) {
            cplx* v = Vt + p * ld;
            for (int i = 0; i < m; ++i) v[i] = cmake(0.0, 0.0);
            v[p] = cmake(1.0, 0.0);
            cplx lp = A[p * ld + p];
            for (int i = p - 1; i >= 0; --i) {
                cplx acc = cmake(0.0, 0.0);
                for (int j = i + 1; j <= p; ++j) cfma(acc, A[i * ld + j], v[j]);
                cplx den = csub(A[i * ld + i], lp);
                if (cabsd(den) < small) den = cmake(small, 0.0);
                v[i] = cscale(cdiv(acc, den), -1.0);
            }
        }
        __syncwarp();
        for (int p = 0; p < m; ++p) {
            const cplx* v = Vt + p * ld;
            double nrm = 0.0;
            cplx yv[2];
            for (int t = 0; t < 2; ++t) {
                int r = lane + 32 * t;
                cplx acc = cmake(0.0, 0.0);
                if (r < m)
                    for (int i = 0; i <= p; ++i) cfma(acc, Z[r * ld + i], v[i]);
                yv[t] = acc;
                nrm += cabs2(acc);
            }
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
            for (int t = 0; t < 2; ++t) {
                int r = lane + 32 * t;
                if (r < m) evecs[(long long)p * m + r] = cscale(yv[t], inv);
            }
        }
    }
    __syncwarp();
    if (Tout)
        for (int e = lane; e < m * m; e += 32) { int i = e / m, j = e % m; Tout[(long long)j * m + i] = A[i * ld + j]; }
    if (Zout)
        for (int e = lane; e < m * m; e += 32) { int i = e / m, j = e % m; Zout[(long long)j * m + i] = Z[i * ld + j]; }
    if (lane == 0 && info) info[0] = stalled;
}

