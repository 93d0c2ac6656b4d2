// Right-preconditioned GMRES (Sec. 3.1, App. A.2), steady-state refinement, shift-invert
// Krylov-Schur Arnoldi for the low-lying spectrum (Alg. 5) and the pure steady state of
// Theorem 1's first case.  Every vector lives in Schur coordinates X~ = Q^dag X Q, where the
// Hilbert-Schmidt inner product is unchanged; the max-norm stopping tests are evaluated in
// the original basis with the FP64 Lindbladian.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <complex>
#include <vector>

#include "lb_internal.cuh"
#include "vecops.cuh"

namespace {

// ---------------------------------------------------------------- small device kernels
// least squares min || beta e1 - Hbar y || for the (k+1) x k Hessenberg Hbar (column-major,
// ld ldh) by Givens rotations; y[0..k-1], res[0] = |residual|.  One thread.
__global__ void k_hess_lstsq(const cplx* Hb, int ldh, int k, double beta, cplx* work, cplx* y, double* res) {
    if (threadIdx.x != 0) return;
    cplx* R = work;                 // (k+1) x k copy, column-major ld k+1
    cplx* g = work + (k + 1) * k;   // k+1
    for (int j = 0; j < k; ++j)
        for (int i = 0; i <= k; ++i) R[j * (k + 1) + i] = (i <= j + 1) ? Hb[(long long)j * ldh + i] : cmake(0, 0);
    for (int i = 0; i <= k; ++i) g[i] = cmake(i == 0 ? beta : 0.0, 0.0);
    for (int j = 0; j < k; ++j) {
        cplx x = R[j * (k + 1) + j], yv = R[j * (k + 1) + j + 1];
        double ax = hypot(x.x, x.y), ay = hypot(yv.x, yv.y);
        double c; cplx s;
        if (ay == 0.0) { c = 1.0; s = cmake(0, 0); }
        else if (ax == 0.0) { c = 0.0; s = cscale(cconj(yv), 1.0 / ay); }
        else { double r = hypot(ax, ay); c = ax / r; s = cscale(cmul(cscale(x, 1.0 / ax), cconj(yv)), 1.0 / r); }
        for (int jj = j; jj < k; ++jj) {
            cplx a = R[jj * (k + 1) + j], b = R[jj * (k + 1) + j + 1];
            R[jj * (k + 1) + j] = cadd(cscale(a, c), cmul(s, b));
            R[jj * (k + 1) + j + 1] = csub(cscale(b, c), cmul(cconj(s), a));
        }
        cplx a = g[j], b = g[j + 1];
        g[j] = cadd(cscale(a, c), cmul(s, b));
        g[j + 1] = csub(cscale(b, c), cmul(cconj(s), a));
    }
    for (int i = k - 1; i >= 0; --i) {
        cplx acc = g[i];
        for (int j = i + 1; j < k; ++j) acc = csub(acc, cmul(R[j * (k + 1) + i], y[j]));
        cplx d = R[i * (k + 1) + i];
        y[i] = (d.x == 0.0 && d.y == 0.0) ? cmake(0, 0) : cdiv(acc, d);
    }
    res[0] = hypot(g[k].x, g[k].y);
}

// Sherman-Morrison combination of Alg. 2: out = Z + coef * W with
// coef = c Tr(Z) / (1 - c Tr W); trz and trw device scalars.
__global__ void k_sm_combine(cplx* out, const cplx* W, long long len, const cplx* trz, const cplx* trw, double c) {
    cplx den = csub(cmake(1.0, 0.0), cscale(trw[0], c));
    cplx coef = cdiv(cscale(trz[0], c), den);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
        out[e] = cadd(out[e], cmul(coef, W[e]));
}

// deterministic traceless start vector: hashed uniform entries, diagonal shifted to trace 0
__global__ void k_start_vector(cplx* X, int n, unsigned seed) {
    long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)e * 0x9E3779B97F4A7C15ull + seed;
        z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 27; z *= 0x94D049BB133111EBull; z ^= z >> 31;
        double a = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        z = z * 0x9E3779B97F4A7C15ull + 1;
        z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 27; z *= 0x94D049BB133111EBull; z ^= z >> 31;
        double b = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        X[e] = cmake(a, b);
    }
}

// Krylov-Schur restart of the small matrices: Hnew[:p,:p] = T[:p,:p]; Hnew[p, j] = beta Zs[m-1, j]
__global__ void k_ks_restart(cplx* Hm, int ldh, const cplx* T, const cplx* Zs, int m, int p) {
    __shared__ cplx beta;
    if (threadIdx.x == 0) beta = Hm[(long long)(m - 1) * ldh + m];
    __syncthreads();
    for (int e = threadIdx.x; e < (KMAX + 1) * (KMAX + 1); e += blockDim.x) {
        int j = e / (KMAX + 1), i = e % (KMAX + 1);
        if (j >= ldh || i >= ldh) continue;
        cplx v = cmake(0, 0);
        if (j < p && i < p) v = T[(long long)j * m + i];
        else if (j < p && i == p) v = cmul(beta, Zs[(long long)j * m + m - 1]);
        Hm[(long long)j * ldh + i] = v;
    }
}

// eigenvector of upper-triangular T for the diagonal entry of smallest |Re| (case 1 of
// Theorem 1): v_p = 1, v_i = -sum_{j=i+1..p} T_ij v_j / (T_ii - T_pp); one CTA.
__global__ void k_case1_vector(const cplx* T, int n, cplx* v) {
    __shared__ int p;
    __shared__ double red[32];
    __shared__ int redi[32];
    __shared__ cplx acc_s[32];
    double best = 1e300;
    int bi = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double a = fabs(T[(long long)i * n + i].x);
        if (a < best) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = best; redi[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 1e300; int ii = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
            if (red[q] < b || (red[q] == b && redi[q] < ii)) { b = red[q]; ii = redi[q]; }
        p = ii;
    }
    __syncthreads();
    const int pp = p;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = cmake(i == pp ? 1.0 : 0.0, 0.0);
    __syncthreads();
    const cplx lp = T[(long long)pp * n + pp];
    for (int i = pp - 1; i >= 0; --i) {
        cplx a = cmake(0, 0);
        for (int j = i + 1 + threadIdx.x; j <= pp; j += blockDim.x) cfma(a, T[(long long)i * n + j], v[j]);
        for (int o = 16; o > 0; o >>= 1) {
            a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
        }
        if ((threadIdx.x & 31) == 0) acc_s[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            cplx t = cmake(0, 0);
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = cadd(t, acc_s[q]);
            cplx den = csub(T[(long long)i * n + i], lp);
            if (hypot(den.x, den.y) < 1e-300) den = cmake(1e-300, 0);
            v[i] = cscale(cdiv(t, den), -1.0);
        }
        __syncthreads();
    }
}

// rho = psi psi^dag / ||psi||^2 (nrm2[0] = ||psi||^2 as the real part)
__global__ void k_outer(cplx* rho, const cplx* psi, int n, const cplx* nrm2) {
    double inv = 1.0 / nrm2[0].x;
    long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / n), j = (int)(e % n);
        rho[e] = cscale(cmul(psi[i], cconj(psi[j])), inv);
    }
}

inline int grid1(long long len) { long long g = (len + 255) / 256; return (int)std::min<long long>(std::max<long long>(g, 1), 1184); }

double read_double(cudaStream_t s, const double* d) {
    double v = NAN;
    cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return v;
}

}  // namespace

// ============================================================================ Alg. 2
// W = R_mu^S(I) in Schur coordinates and its trace (scal[8]); returns LB_ETA_EXCLUDED if
// |1 - eta Tr W| is negligible (Eq. ShermanMorr).
lb_status precond_prepare(lb_handle_s* h, cudaStream_t s, double mu, double eta, int precision, int adj) {
    const int n = h->n;
    cplx* W = adj ? h->Wa : h->W;
    // (mu - S~) W = I  <=>  T_mu W + W T_mu^dag = -I   (adjoint: T_mu^dag W + W T_mu = -I)
    if (mat_eye(W, n, cmake(-1, 0), s)) return LB_CUDA_ERROR;
    if (adj ? adj_lyap_schur(h, s, W, W, 0.5 * mu) : lyap_schur(h, s, W, W, 0.5 * mu, precision))
        return LB_CUDA_ERROR;
    if (mat_trace(W, n, h->scal + 8, s)) return LB_CUDA_ERROR;
    cplx trw;
    LB_CHECK_CUDA(cudaMemcpyAsync(&trw, h->scal + 8, sizeof(cplx), cudaMemcpyDeviceToHost, s));
    LB_CHECK_CUDA(cudaStreamSynchronize(s));
    std::complex<double> den = 1.0 - eta * std::complex<double>(trw.x, trw.y);
    if (std::abs(den) < 1e-8) return LB_ETA_EXCLUDED;
    return LB_OK;
}

// out = Precond(X, mu, eta) = Z + eta Tr Z / (1 - eta Tr W) W, Z = R_mu^S(X)  (Alg. 2); with eta = 0
// it is the plain no-jump resolvent R_mu^S (the preconditioner of the undeflated systems) and W is
// not read
int precond_apply(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* out, double mu, double eta, int precision,
                  int adj) {
    const long long nn = (long long)h->n * h->n;
    if (vec_scale_copy(out, X, nn, cmake(-1, 0), s)) return -1;                // -X
    if (adj ? adj_lyap_schur(h, s, out, out, 0.5 * mu) : lyap_schur(h, s, out, out, 0.5 * mu, precision))
        return -1;                                                               // Z
    if (eta == 0.0) return 0;
    if (mat_trace(out, h->n, h->scal + 9, s)) return -1;
    k_sm_combine<<<grid1(nn), 256, 0, s>>>(out, adj ? h->Wa : h->W, nn, h->scal + 9, h->scal + 8, eta); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// out = (mu - L~_eta)(X) = mu X - (T X + X T^dag) - K~(X) - eta Tr(X) I   (Schur coordinates)
static int shifted_deflated_apply(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* out, double mu, double eta,
                                  int precision) {
    const int n = h->n;
    const long long nn = (long long)n * n;
    if (gemm(h, s, out, h->T, OP_N, X, OP_N, n, n, n, cmake(-1, 0), cmake(0, 0))) return -1;
    if (gemm(h, s, out, X, OP_N, h->T, OP_C, n, n, n, cmake(-1, 0), cmake(1, 0))) return -1;
    if (precision == LB_PREC_MIXED && h->mixed_ready) {
        if (jump_mixed(h, s, X, h->X[7], 1.0)) return -1;
        if (vec_axpby(out, h->X[7], nn, cmake(-1, 0), cmake(1, 0), s)) return -1;
    } else if (jump_f64(h, s, h->Lt, X, out, cmake(-1, 0), cmake(1, 0))) {
        return -1;
    }
    if (vec_axpby(out, X, nn, cmake(mu, 0), cmake(1, 0), s)) return -1;
    if (mat_trace(X, n, h->scal + 10, s)) return -1;
    return mat_add_diag_dev(out, n, h->scal + 10, -eta, s);
}

// residual coefficients after a GMRES cycle: g = beta e1 - Hbar y ((k+1)-vector), so that the new
// residual is V_{k+1} g (Arnoldi relation A P V_k = V_{k+1} Hbar)
__global__ void k_gmres_resid_coeffs(const cplx* Hb, int ldh, int k, double beta, const cplx* y, cplx* g) {
    for (int i = threadIdx.x; i <= k; i += blockDim.x) {
        cplx acc = cmake(i == 0 ? beta : 0.0, 0.0);
        for (int j = (i > 0 ? i - 1 : 0); j < k; ++j) acc = csub(acc, cmul(Hb[(long long)j * ldh + i], y[j]));
        g[i] = acc;
    }
}

// Restarted right-preconditioned GMRES(m) for (mu - L~_eta) x = b in Schur coordinates, from
// x = 0, preconditioner P = Precond(., mu, eta).  Because P inverts (mu - S~) - eta |I><I| exactly
// (Sherman-Morrison), the preconditioned operator is (mu - L~_eta) P = Id - K~ P (the right-
// preconditioning identity of Sec. 3.1): one Lyapunov solve and one jump term per step, no
// application of S~.  Residuals between cycles follow from the Arnoldi relation.  Stops when the
// residual norm <= atol, on stagnation (< 10% gain per cycle) or after max_cycles.
// Uses V / hm (inner basis), X[5], X[6], X[7].
static int gmres_solve(lb_handle_s* h, cudaStream_t s, const cplx* b, cplx* x, double mu, double eta, int m,
                       int max_cycles, double atol, int precision, int* steps, double* final_res, int adj = 0) {
    const long long nn = (long long)h->n * h->n;
    cplx* r = h->X[5];
    cplx* pv = h->X[6];
    cplx* y = h->small + 3 * (KMAX + 2);
    cplx* g = h->ev;   // (k+1) residual coefficients
    double* dres = h->dscal + 6;
    OpFn op = [&](const cplx* v, cplx* w) {
        if (precond_apply(h, s, v, pv, mu, eta, precision, adj)) return -1;
        if (adj) {
            if (adj_jump_f64(h, s, pv, w, cmake(-1, 0), cmake(0, 0))) return -1;
        } else if (precision == LB_PREC_MIXED && h->mixed_ready) {
            if (jump_mixed(h, s, pv, w, -1.0)) return -1;
        } else if (jump_f64(h, s, h->Lt, pv, w, cmake(-1, 0), cmake(0, 0))) {
            return -1;
        }
        return vec_axpby(w, v, nn, cmake(1, 0), cmake(1, 0), s);
    };
    if (vec_scale_copy(x, b, nn, cmake(0, 0), s)) return -1;
    if (vec_scale_copy(r, b, nn, cmake(1, 0), s)) return -1;
    if (vec_norms(r, nn, h->dpart, h->dscal, s)) return -1;
    double beta = read_double(s, h->dscal + 1);
    double res = beta;
    for (int cyc = 0; cyc < max_cycles && beta > atol; ++cyc) {
        if (vec_scale_copy(h->V, r, nn, cmake(1.0 / beta, 0), s)) return -1;
        int k = 0;
        if (arnoldi_cycle(h, s, h->V, h->hm, 0, m, op, &k)) return -1;
        *steps += k;
        k_hess_lstsq<<<1, 32, 0, s>>>(h->hm, h->ldh, k, beta, h->evec, y, dres); lb_note_launch();
        if (vec_gemv(r, h->V, nn, k, y, nn, 1.0, 0, s)) return -1;           // u = V y
        if (precond_apply(h, s, r, pv, mu, eta, precision, adj)) return -1;   // P u
        if (vec_axpby(x, pv, nn, cmake(1, 0), cmake(1, 0), s)) return -1;  // x += P u
        k_gmres_resid_coeffs<<<1, 64, 0, s>>>(h->hm, h->ldh, k, beta, y, g); lb_note_launch();
        if (vec_gemv(r, h->V, nn, k + 1, g, nn, 1.0, 0, s)) return -1;      // r = V_{k+1} g
        const double prev = beta;
        beta = read_double(s, dres);
        res = beta;
        if (beta > 0.9 * prev) break;   // stagnation
    }
    *final_res = res;
    return 0;
}

// entry points for the adjoint solve (adjoint.cu)
lb_status adj_precond_prepare(lb_handle_s* h, cudaStream_t s, double eta) {
    return precond_prepare(h, s, 0.0, eta, LB_PREC_FP64, 1);
}
int adj_gmres_solve(lb_handle_s* h, cudaStream_t s, const cplx* b, cplx* x, double eta, int m, int max_cycles,
                    double atol, int* steps, double* final_res) {
    return gmres_solve(h, s, b, x, 0.0, eta, m, max_cycles, atol, LB_PREC_FP64, steps, final_res, 1);
}

// ============================================================================ case 1
int pure_state_case1(lb_handle_s* h, cudaStream_t s, cplx* rho_out) {
    const int n = h->n;
    cplx* v = h->X[0];
    cplx* psi = h->X[1];
    k_case1_vector<<<1, 256, 0, s>>>(h->T, n, v); lb_note_launch();
    if (gemm(h, s, psi, h->Q, OP_N, v, OP_N, n, 1, n, cmake(1, 0), cmake(0, 0))) return -1;
    if (vec_dot_block(psi, n, 1, psi, n, h->scal + 3, h->part, 0, s)) return -1;
    k_outer<<<grid1((long long)n * n), 256, 0, s>>>(rho_out, psi, n, h->scal + 3); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ============================================================================ refinement
// Residual correction of the steady state (mixed precision).  The state is kept in Schur coordinates
// (rs = h->best, Hermitian, trace 1) with its residual R~ = Q^dag L(rho) Q.  Each step solves
// (0 - L~_eta) delta = R~ approximately by preconditioned GMRES (Alg. 3's operator, Alg. 2's
// preconditioner at lambda = 0) on the tensor cores, applies the hermitised correction d, and updates
// the residual by linearity, R~ <- (R~ + T d + (T d)^dag + K~(d)) / t (t the new trace): one FP64 GEMM and
// a tensor-core jump term instead of a full FP64 Lindbladian.  The error of that update is of the
// order of the tensor-core precision times ||K~ d||, far below the tolerance near convergence; the
// state is certified by an exact FP64 residual in the original basis when ||R~||_F (an upper bound
// on the max-norm) falls below the tolerance, when the estimate stagnates, or at the step cap.  A
// certified residual that is not lower than the previous one undoes the steps since the last
// certification, so the returned state is always the best one certified (the running best of Alg. 4).
// On entry h->Rres holds L(rho) of rho (original basis, written by the Arnoldi phase); on return it
// holds the last certified residual (which may belong to a rejected step).
lb_status refine_steady_state(lb_handle_s* h, cudaStream_t s, const lb_opts& o, cplx* rho, lb_info* inf) {
    const int n = h->n;
    const long long nn = (long long)n * n;
    const size_t bytes = (size_t)nn * sizeof(cplx);
    lb_status st = precond_prepare(h, s, 0.0, o.eta, o.precision, 0);
    if (st != LB_OK) return st;
    const bool mixed = o.precision == LB_PREC_MIXED && h->mixed_ready;
    cplx* Rt = h->X[1];     // residual estimate in Schur coordinates
    cplx* A = h->X[2];
    cplx* delta = h->X[3];
    cplx* dh = h->X[4];
    cplx* Kd = h->X[0];
    cplx* rs = h->best;     // Schur-coordinate state
    double rmax = inf->residual_max, rfro = inf->residual_fro;
    if (change_basis(h, s, h->Rres, Rt, A, 1)) return LB_CUDA_ERROR;
    LB_CHECK_CUDA(cudaMemcpyAsync(h->bk0, rho, bytes, cudaMemcpyDeviceToDevice, s));
    LB_CHECK_CUDA(cudaMemcpyAsync(h->bk1, rs, bytes, cudaMemcpyDeviceToDevice, s));
    double est = rfro, prev_est = INFINITY;
    for (int it = 0; it < o.max_refine && rmax >= o.tol; ++it) {
        if (vec_scale_copy(delta, Rt, nn, cmake(0, 0), s)) return LB_CUDA_ERROR;
        int steps = 0;
        double res = 0.0;
        if (gmres_solve(h, s, Rt, delta, 0.0, o.eta, o.gmres_m, 3, 1e-6 * est, o.precision, &steps, &res))
            return LB_CUDA_ERROR;
        inf->gmres_steps += steps;
        inf->refine_steps += 1;
        // d = herm(delta); R~ += T d + (T d)^dag + K~(d); rs += d; both divided by t = Tr(rs)
        if (mat_hermitize(dh, delta, n, s)) return LB_CUDA_ERROR;
        if (gemm(h, s, A, h->T, OP_N, dh, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return LB_CUDA_ERROR;
        if (mat_add_adjoint(A, n, s)) return LB_CUDA_ERROR;
        if (mixed ? jump_mixed(h, s, dh, Kd, 1.0, 1) : jump_f64(h, s, h->Lt, dh, Kd, cmake(1, 0), cmake(0, 0), 1))
            return LB_CUDA_ERROR;
        if (vec_axpby(Rt, A, nn, cmake(1, 0), cmake(1, 0), s)) return LB_CUDA_ERROR;
        if (vec_axpby(Rt, Kd, nn, cmake(1, 0), cmake(1, 0), s)) return LB_CUDA_ERROR;
        if (vec_axpby(rs, dh, nn, cmake(1, 0), cmake(1, 0), s)) return LB_CUDA_ERROR;
        if (mat_trace(rs, n, h->scal + 1, s)) return LB_CUDA_ERROR;
        if (mat_div_by_dev(rs, rs, nn, h->scal + 1, s, 1)) return LB_CUDA_ERROR;
        if (mat_div_by_dev(Rt, Rt, nn, h->scal + 1, s, 1)) return LB_CUDA_ERROR;
        if (vec_norms(Rt, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
        double nr[2];
        LB_CHECK_CUDA(cudaMemcpyAsync(nr, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaStreamSynchronize(s));
        prev_est = est;
        est = nr[1];
        const bool certify = est < o.tol || !(est < 0.3 * prev_est) || it + 1 == o.max_refine;
        if (!certify) continue;
        // exact FP64 residual of the state in the original basis
        if (change_basis(h, s, rs, rho, A, 0)) return LB_CUDA_ERROR;
        if (hermitize_normalize(h, s, rho, rho, A)) return LB_CUDA_ERROR;
        double nmax = 0.0, nfro = 0.0;
        if (residual_norms(h, s, rho, h->Rres, &nmax, &nfro)) return LB_CUDA_ERROR;
        if (!(nmax < rmax)) {
            // no progress (the correction hit the low-precision floor): back to the certified state
            LB_CHECK_CUDA(cudaMemcpyAsync(rho, h->bk0, bytes, cudaMemcpyDeviceToDevice, s));
            LB_CHECK_CUDA(cudaMemcpyAsync(rs, h->bk1, bytes, cudaMemcpyDeviceToDevice, s));
            break;
        }
        rmax = nmax;
        rfro = nfro;
        LB_CHECK_CUDA(cudaMemcpyAsync(h->bk0, rho, bytes, cudaMemcpyDeviceToDevice, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(h->bk1, rs, bytes, cudaMemcpyDeviceToDevice, s));
        if (rmax >= o.tol) {
            // continue from the exact residual
            if (change_basis(h, s, h->Rres, Rt, A, 1)) return LB_CUDA_ERROR;
            est = rfro;
        }
    }
    LB_CHECK_CUDA(cudaStreamSynchronize(s));
    inf->residual_max = rmax;
    inf->residual_fro = rfro;
    return rmax < o.tol ? LB_OK : LB_NOT_CONVERGED;
}

// ============================================================================ Alg. 5
static lb_status low_spectrum_body(lindblad_handle h, int k, double mu, double eta, void* evals_host, void* evecs_dev,
                                  const lb_opts* opts, lb_info* info, void* stream) {
    if (!h || !evals_host) return LB_INVALID_ARG;
    lb_opts o = h->opts;
    if (opts) o = *opts;
    const int m = o.krylov_m;
    if (k < 1 || m < k + 2 || m + 1 > h->vcap || m > KMAX || o.gmres_m + 1 > h->vcap) return LB_INVALID_ARG;
    if (h->case1 && !(mu > 0.0)) return LB_S_SINGULAR;
    if (o.precision == LB_PREC_MIXED && !h->mixed_ready) return LB_NOT_IMPLEMENTED;
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const int n = h->n;
    const long long nn = (long long)n * n;
    int p = o.keep_ritz > 0 ? o.keep_ritz : std::max(k + 2, std::min(m - 2, 2 * k));
    p = std::min(std::max(p, k), m - 1);
    lb_info inf{};
    inf.schur_backward_err = h->schur_err;
    inf.min_abs_re_T = h->min_re_T;
    inf.setup_ms = h->setup_ms;
    lb_status st = precond_prepare(h, s, mu, eta, o.precision, 0);
    if (st != LB_OK) return st;
    // the outer relation matrix is read as a general matrix by the small Schur kernel: clear it
    LB_CHECK_CUDA(cudaMemsetAsync(h->hm2, 0, (size_t)(KMAX + 1) * (KMAX + 1) * sizeof(cplx), s));
    // start vector: traceless, unit norm
    cplx* Zb = h->Z;
    k_start_vector<<<grid1(nn), 256, 0, s>>>(Zb, n, 12345u); lb_note_launch();
    if (mat_trace(Zb, n, h->scal + 4, s)) return LB_CUDA_ERROR;
    if (mat_add_diag_dev(Zb, n, h->scal + 4, -1.0 / n, s)) return LB_CUDA_ERROR;
    if (vec_norms(Zb, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
    double z0 = read_double(s, h->dscal + 1);
    if (vec_scale_copy(Zb, Zb, nn, cmake(1.0 / z0, 0), s)) return LB_CUDA_ERROR;

    cplx* xsol = h->X[4];
    std::vector<cplx> evh(KMAX), lam(k);
    std::vector<double> resid(k, INFINITY);
    // the small ordered Schur form (T, Zs), Ritz values and vectors: carved from the dot-product
    // partial buffer (DOT_BLOCKS (KMAX+2) entries >> 3 KMAX^2); copied to host right away
    // because the next OP call reuses that buffer
    cplx* Ts = h->part;
    cplx* Zs = h->part + (size_t)KMAX * KMAX;
    cplx* evs = h->part + (size_t)2 * KMAX * KMAX;
    cplx* evv = h->part + (size_t)2 * KMAX * KMAX + KMAX;
    int j0 = 0, restart = 0;
    double worst = INFINITY;
    // mixed precision: the inner solves run on the tensor cores while the eigen-residual falls, then in
    // FP64 (W recomputed in FP64) after an explicit restart from the wanted Schur vectors
    int prec = o.precision;
    double prev_worst = INFINITY;
    const bool verbose = std::getenv("LB_VERBOSE") != nullptr;   // diagnostics on stderr, no effect on results
    OpFn OP = [&](const cplx* b, cplx* x) {
        // x = (mu - L~_eta)^{-1} b by preconditioned GMRES, zero initial guess
        if (vec_scale_copy(xsol, b, nn, cmake(0, 0), s)) return -1;
        double bn = 0.0;
        if (vec_norms(b, nn, h->dpart, h->dscal, s)) return -1;
        bn = read_double(s, h->dscal + 1);
        if (!std::isfinite(bn)) return -1;
        int steps = 0;
        double res = 0.0;
        if (gcrodr_solve(h, s, b, xsol, mu, eta, o.gmres_m, o.recycle_k, 50, o.inner_tol * bn, prec, &steps, &res,
                         nullptr))
            return -1;
        // the recycled pair makes the GMRES estimate a statement about B U = C: check the true residual
        // b - (mu - L~_eta) x with one explicit application; if it disagrees, drop the pair and continue
        // the solve from the true residual with plain cycles
        for (int attempt = 0; attempt < 2; ++attempt) {
            cplx* Ax = h->X[2];
            cplx* corr = h->X[3];
            if (shifted_deflated_apply(h, s, xsol, Ax, mu, eta, prec)) return -1;
            if (vec_axpby(Ax, b, nn, cmake(1, 0), cmake(-1, 0), s)) return -1;   // Ax <- b - A x
            if (vec_norms(Ax, nn, h->dpart, h->dscal, s)) return -1;
            const double tr = read_double(s, h->dscal + 1);
            if (!std::isfinite(tr)) return -1;
            const double floor_mixed = prec == LB_PREC_MIXED ? 1e-5 * bn : 0.0;
            if (!(tr > 10.0 * std::max(std::max(res, o.inner_tol * bn), floor_mixed))) break;
            if (verbose) fprintf(stderr, "  OP %d: true residual %.2e against the estimate %.2e: pair dropped\n",
                                 inf.phi_applies + 1, tr / bn, res / bn);
            recycle_forget(h);
            int st2 = 0;
            if (gcrodr_solve(h, s, Ax, corr, mu, eta, o.gmres_m, o.recycle_k, 50, o.inner_tol * bn, prec, &st2, &res,
                             nullptr))
                return -1;
            steps += st2;
            if (vec_axpby(xsol, corr, nn, cmake(1, 0), cmake(1, 0), s)) return -1;
        }
        inf.gmres_steps += steps;
        inf.phi_applies += 1;
        if (verbose) fprintf(stderr, "  OP %d: %d inner steps, relative residual %.2e\n", inf.phi_applies, steps, res / bn);
        return vec_scale_copy(x, xsol, nn, cmake(1, 0), s);
    };
    // small results must not be overwritten by the GMRES of the next OP call: part is used by
    // vec_dot_block, so copy them to host-side mirrors right after each small_schur
    std::vector<cplx> Th((size_t)m * m), Zh((size_t)m * m), Yh((size_t)m * m);
    for (; restart < o.max_restarts; ++restart) {
        int kk = 0;
        if (arnoldi_cycle(h, s, Zb, h->hm2, j0, m, OP, &kk)) return LB_CUDA_ERROR;
        const int mm = kk;
        if (mm < k) { st = LB_NOT_CONVERGED; break; }
        if (small_schur(h->hm2, h->ldh, mm, 0, 1, std::min(p, mm), evs, evv, Ts, Zs, h->dinfo, s))
            return LB_CUDA_ERROR;
        LB_CHECK_CUDA(cudaMemcpyAsync(evh.data(), evs, mm * sizeof(cplx), cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(Yh.data(), evv, (size_t)mm * mm * sizeof(cplx), cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(Th.data(), Ts, (size_t)mm * mm * sizeof(cplx), cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(Zh.data(), Zs, (size_t)mm * mm * sizeof(cplx), cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaStreamSynchronize(s));
        // Ritz pairs: the k leading (largest |nu|) of the ordered Schur form
        worst = 0.0;
        for (int i = 0; i < k; ++i) {
            std::complex<double> nu(evh[i].x, evh[i].y);
            std::complex<double> l = mu - 1.0 / nu;
            lam[i] = cmake(l.real(), l.imag());
            // v_i = Zb y_i (Schur coordinates) -> original basis -> ||L v - lam v||_max / ||v||_max
            LB_CHECK_CUDA(cudaMemcpyAsync(h->small, Yh.data() + (size_t)i * mm, mm * sizeof(cplx),
                                          cudaMemcpyHostToDevice, s));
            cplx* vt = h->X[5];
            cplx* v = h->X[6];
            cplx* R = h->X[7];
            if (vec_gemv(vt, Zb, nn, mm, h->small, nn, 1.0, 0, s)) return LB_CUDA_ERROR;
            if (change_basis(h, s, vt, v, R, 0)) return LB_CUDA_ERROR;
            if (evecs_dev) {
                LB_CHECK_CUDA(cudaMemcpyAsync((cplx*)evecs_dev + (size_t)i * nn, v, nn * sizeof(cplx),
                                              cudaMemcpyDeviceToDevice, s));
            }
            if (lindbladian_f64(h, s, v, R)) return LB_CUDA_ERROR;
            if (vec_axpby(R, v, nn, cmake(-l.real(), -l.imag()), cmake(1, 0), s)) return LB_CUDA_ERROR;
            if (vec_norms(R, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
            if (vec_norms(v, nn, h->dpart, h->dscal + 2, s)) return LB_CUDA_ERROR;
            double nr[4];
            LB_CHECK_CUDA(cudaMemcpyAsync(nr, h->dscal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
            LB_CHECK_CUDA(cudaStreamSynchronize(s));
            resid[i] = nr[0] / std::max(nr[2], 1e-300);
            worst = std::max(worst, resid[i]);
        }
        inf.restarts = restart + 1;
        inf.residual_max = worst;
        if (verbose)
            fprintf(stderr, "low_spectrum: cycle %d size %d precision %d worst eigen-residual %.3e, lambda_1 = %.6e %+.6ei, "
                            "inner steps so far %d\n",
                    restart, mm, prec, worst, lam[0].x, lam[0].y, inf.gmres_steps);
        if (worst < o.tol) { st = LB_OK; break; }
        if (prec == LB_PREC_FP64 && o.precision == LB_PREC_MIXED) inf.refine_steps += 1;
        if (prec == LB_PREC_MIXED && (worst < 1e-6 || !(worst < 0.5 * prev_worst))) {
            prec = LB_PREC_FP64;
            st = precond_prepare(h, s, mu, eta, LB_PREC_FP64, 0);
            if (st != LB_OK) return st;
            // explicit restart: a thick restart would keep the tensor-core OP images in the Krylov-Schur
            // relation and bound every later Ritz pair at that precision; the FP64 cycles start from the
            // sum of the k wanted Schur vectors (orthonormal, so no cancellation), which holds the
            // wanted eigenvectors to the mixed accuracy
            std::vector<cplx> y((size_t)mm, cmake(0, 0));
            for (int j = 0; j < k; ++j)
                for (int i = 0; i < mm; ++i) {
                    y[i].x += Zh[(size_t)j * mm + i].x;
                    y[i].y += Zh[(size_t)j * mm + i].y;
                }
            LB_CHECK_CUDA(cudaMemcpyAsync(h->small, y.data(), mm * sizeof(cplx), cudaMemcpyHostToDevice, s));
            if (vec_gemv(h->V, Zb, nn, mm, h->small, nn, 1.0, 0, s)) return LB_CUDA_ERROR;
            if (vec_norms(h->V, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
            const double z1 = read_double(s, h->dscal + 1);
            if (!(z1 > 0.0) || !std::isfinite(z1)) return LB_CUDA_ERROR;
            if (vec_scale_copy(Zb, h->V, nn, cmake(1.0 / z1, 0), s)) return LB_CUDA_ERROR;
            LB_CHECK_CUDA(cudaMemsetAsync(h->hm2, 0, (size_t)(KMAX + 1) * (KMAX + 1) * sizeof(cplx), s));
            j0 = 0;
            prev_worst = INFINITY;
            st = LB_NOT_CONVERGED;
            continue;
        }
        prev_worst = std::min(prev_worst, worst);
        if (mm < m) { st = LB_NOT_CONVERGED; break; }   // invariant subspace smaller than m: cannot restart
        // thick restart: Zb[:p] <- Zb Zs[:, :p]; Zb[p] <- Zb[m]; H <- [T_pp; beta Zs[m-1, :p]]
        LB_CHECK_CUDA(cudaMemcpyAsync(Zs, Zh.data(), (size_t)mm * mm * sizeof(cplx), cudaMemcpyHostToDevice, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(Ts, Th.data(), (size_t)mm * mm * sizeof(cplx), cudaMemcpyHostToDevice, s));
        for (int j = 0; j < p; ++j)
            if (vec_gemv(h->V + (size_t)j * nn, Zb, nn, mm, Zs + (size_t)j * mm, nn, 1.0, 0, s))
                return LB_CUDA_ERROR;
        LB_CHECK_CUDA(cudaMemcpyAsync(Zb, h->V, (size_t)p * nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(Zb + (size_t)p * nn, Zb + (size_t)mm * nn, nn * sizeof(cplx),
                                      cudaMemcpyDeviceToDevice, s));
        k_ks_restart<<<1, 256, 0, s>>>(h->hm2, h->ldh, Ts, Zs, mm, p); lb_note_launch();
        j0 = p;
        st = LB_NOT_CONVERGED;
    }
    // sort the k values by |lambda|, then Re descending, then Im ascending
    std::vector<int> idx(k);
    for (int i = 0; i < k; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) {
        double ma = std::hypot(lam[a].x, lam[a].y), mb = std::hypot(lam[b].x, lam[b].y);
        if (std::fabs(ma - mb) > 1e-12 * std::max(ma, mb)) return ma < mb;
        if (lam[a].x != lam[b].x) return lam[a].x > lam[b].x;
        return lam[a].y < lam[b].y;
    });
    cplx* outv = (cplx*)evals_host;
    for (int i = 0; i < k; ++i) outv[i] = lam[idx[i]];
    if (evecs_dev) {
        // permute the stored eigenvectors to the sorted order (via the V scratch)
        for (int i = 0; i < k; ++i)
            LB_CHECK_CUDA(cudaMemcpyAsync(h->V + (size_t)i * nn, (cplx*)evecs_dev + (size_t)idx[i] * nn,
                                          nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(evecs_dev, h->V, (size_t)k * nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    }
    LB_CHECK_CUDA(cudaStreamSynchronize(s));
    inf.status = st;
    inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return st;
}

extern "C" lb_status low_spectrum(lindblad_handle h, int k, double mu, double eta, void* evals_host, void* evecs_dev,
                                  const lb_opts* opts, lb_info* info, void* stream) {
    return device_error_guard(h, (cudaStream_t)stream, low_spectrum_body(h, k, mu, eta, evals_host, evecs_dev, opts, info, stream));
}
