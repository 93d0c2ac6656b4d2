// Implicit differentiation of the steady state (Remark "Differentiating the steady state").
//
// With L~_eta rho = eta I and a real figure of merit J = Re Tr(O rho) (O Hermitian), the gradient
// is dJ = -Re <w, (dL) rho>, where the adjoint state w solves the single system
//     L~_eta^* w = O,   L~_eta^*(w) = G^dag w + w G + sum_j L_j^dag w L_j + eta Tr(w) I.
// The same no-jump preconditioner applies: (mu - S^*) is again a Lyapunov operator,
// S^*(X) = G^dag X + X G, which in Schur coordinates reads T^dag X~ + X~ T = Y~.  With J the index
// reversal, U = J T^dag J is upper triangular and T^dag X~ + X~ T = Y~ is U Z + Z U^dag = J Y~ J
// with X~ = J Z J, so the forward triangular solver serves unchanged.
//
// The library returns the sensitivity matrices G_H, G_L[j] with dJ = Re<G_H, dH> + sum_j
// Re<G_L[j], dL_j> (<A, B> = Tr(A^dag B)):
//     G_H   = i (rho w - w rho),
//     G_L_j = -Ws L_j rho + 1/2 L_j (Ws rho + rho Ws),   Ws = w + w^dag,
// so that any parameterisation H(theta), L_j(theta) is differentiated by one contraction.
#include "lb_internal.cuh"
#include "vecops.cuh"

namespace {

// X = J Y J (X[i][j] = Y[n-1-i][n-1-j]); X and Y must differ
__global__ void k_flip(cplx* __restrict__ X, const cplx* __restrict__ Y, int n) {
    const long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        X[e] = Y[(long long)(n - 1 - i) * n + (n - 1 - j)];
    }
}

// U = J T^dag J
__global__ void k_flip_adjoint(cplx* __restrict__ U, const cplx* __restrict__ T, int n) {
    const long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        // (T^dag)[n-1-i][n-1-j] = conj(T[n-1-j][n-1-i])
        U[e] = cconj(T[(long long)(n - 1 - j) * n + (n - 1 - i)]);
    }
}

// Ws = w + w^dag
__global__ void k_herm_sum(cplx* __restrict__ Ws, const cplx* __restrict__ w, int n) {
    const long long len = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        Ws[e] = cadd(w[e], cconj(w[(long long)j * n + i]));
    }
}

inline int grid1(long long len) {
    long long g = (len + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 1184 ? 1184 : g));
}

int flip(cplx* X, const cplx* Y, int n, cudaStream_t s) {
    k_flip<<<grid1((long long)n * n), 256, 0, s>>>(X, Y, n); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

// X solves (T - shift)^dag X + X (T - shift) = Y in Schur coordinates (X may equal Y)
int adj_lyap_schur(lb_handle_s* h, cudaStream_t s, const cplx* Y, cplx* X, double shift) {
    const int n = h->n;
    if (!h->ua_ready) {
        k_flip_adjoint<<<grid1((long long)n * n), 256, 0, s>>>(h->Ua, h->T, n); lb_note_launch();
        h->ua_ready = true;
    }
    cplx* tmp = h->X[1];
    if (tmp == Y || tmp == X) tmp = h->X[2];
    if (flip(tmp, Y, n, s)) return -1;                                   // Z-equation right-hand side
    if (trisylv_f64(h->Ua, tmp, n, cmake(shift, 0.0), s)) return -1;    // U Z + Z U^dag = J Y J
    return flip(X, tmp, n, s);                                           // X = J Z J
}

// Y = alpha sum_j L~_j^dag Z L~_j + beta Y  (Schur coordinates, FP64)
int adj_jump_f64(lb_handle_s* h, cudaStream_t s, const cplx* Z, cplx* Y, cplx alpha, cplx beta) {
    const int n = h->n, d = h->d;
    const long long nn = (long long)n * n;
    ZGemmArgs a{};
    a.M = n; a.N = n; a.K = n;
    a.A = h->Lt; a.lda = n; a.strideA = nn; a.opA = OP_C;          // P_j = L~_j^dag Z
    a.B = Z; a.ldb = n; a.strideB = 0; a.opB = OP_N;
    a.C = h->P; a.ldc = n; a.strideC = nn;
    a.alpha = cmake(1, 0); a.beta = cmake(0, 0); a.batch = d; a.reduce = 0;
    prof_begin(h, s, 1);
    if (zgemm_f64(a, s)) return -1;
    prof_end(h, s, 1, 8.0 * n * (double)n * n * d);
    a.A = h->P; a.strideA = nn; a.opA = OP_N;                        // Y = alpha sum_j P_j L~_j + beta Y
    a.B = h->Lt; a.strideB = nn; a.opB = OP_N;
    a.C = Y; a.strideC = 0;
    a.alpha = alpha; a.beta = beta; a.reduce = 1;
    prof_begin(h, s, 1);
    const int r = zgemm_f64(a, s);
    prof_end(h, s, 1, 8.0 * n * (double)n * n * d);
    return r;
}

// R = L~_eta^*(w) - O in FP64, original basis; returns max and Frobenius norms
static int adjoint_residual(lb_handle_s* h, cudaStream_t s, const cplx* w, const cplx* O, double eta, cplx* R,
                            double* rmax, double* rfro) {
    const int n = h->n, d = h->d;
    const long long nn = (long long)n * n;
    if (gemm(h, s, R, h->G, OP_C, w, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    if (gemm(h, s, R, w, OP_N, h->G, OP_N, n, n, n, cmake(1, 0), cmake(1, 0))) return -1;
    ZGemmArgs a{};
    a.M = n; a.N = n; a.K = n;
    a.A = h->L; a.lda = n; a.strideA = nn; a.opA = OP_C;
    a.B = w; a.ldb = n; a.strideB = 0; a.opB = OP_N;
    a.C = h->P; a.ldc = n; a.strideC = nn;
    a.alpha = cmake(1, 0); a.beta = cmake(0, 0); a.batch = d; a.reduce = 0;
    if (zgemm_f64(a, s)) return -1;
    a.A = h->P; a.opA = OP_N;
    a.B = h->L; a.strideB = nn; a.opB = OP_N;
    a.C = R; a.strideC = 0;
    a.beta = cmake(1, 0); a.reduce = 1;
    if (zgemm_f64(a, s)) return -1;
    if (mat_trace(w, n, h->scal + 11, s)) return -1;
    if (mat_add_diag_dev(R, n, h->scal + 11, eta, s)) return -1;
    if (vec_axpby(R, O, nn, cmake(-1, 0), cmake(1, 0), s)) return -1;
    if (vec_norms(R, nn, h->dpart, h->dscal, s)) return -1;
    double nr[2];
    if (cudaMemcpyAsync(nr, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    *rmax = nr[0];
    *rfro = nr[1];
    return 0;
}

static lb_status steady_state_adjoint_body(lindblad_handle h, const void* rho_dev, const void* O_dev, void* w_dev,
                                          void* gH_dev, void* gL_dev, const lb_opts* opts, lb_info* info,
                                          void* stream) {
    if (!h || !rho_dev || !O_dev || !w_dev) return LB_INVALID_ARG;
    if (h->case1) return LB_S_SINGULAR;
    lb_opts o = h->opts;
    if (opts) o = *opts;
    if (o.gmres_m < 2 || o.gmres_m + 1 > h->vcap || o.gmres_m > KMAX) return LB_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->n, d = h->d;
    const long long nn = (long long)n * n;
    const cplx* rho = (const cplx*)rho_dev;
    const cplx* O = (const cplx*)O_dev;
    cplx* w = (cplx*)w_dev;
    lb_info inf{};
    inf.schur_backward_err = h->schur_err;
    inf.min_abs_re_T = h->min_re_T;
    inf.setup_ms = h->setup_ms;
    lb_status st = adj_precond_prepare(h, s, o.eta);
    if (st != LB_OK) return st;
    // (0 - L~_eta^*) w = -O in Schur coordinates, refined against the FP64 residual
    cplx* b = h->X[3];
    cplx* wt = h->X[4];
    cplx* dw = h->best;
    double rmax = INFINITY, rfro = INFINITY;
    if (vec_scale_copy(wt, O, nn, cmake(0, 0), s)) return LB_CUDA_ERROR;
    if (vec_scale_copy(w, O, nn, cmake(0, 0), s)) return LB_CUDA_ERROR;
    if (vec_scale_copy(h->X[0], O, nn, cmake(-1, 0), s)) return LB_CUDA_ERROR;   // residual of w = 0
    cplx* R = h->X[0];
    for (int it = 0; it < 4; ++it) {
        // R = L~^* w - O (original basis); solve (0 - L~^*) dw = R, i.e. L~^* (w + dw) = O
        if (it > 0 && adjoint_residual(h, s, w, O, o.eta, R, &rmax, &rfro)) return LB_CUDA_ERROR;
        if (it > 0 && rmax < o.tol) break;
        if (change_basis(h, s, R, b, h->X[2], 1)) return LB_CUDA_ERROR;
        if (vec_norms(b, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
        double bn = 0.0;
        if (cudaMemcpyAsync(&bn, h->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return LB_CUDA_ERROR;
        int steps = 0;
        double res = 0.0;
        if (adj_gmres_solve(h, s, b, dw, o.eta, o.gmres_m, 20, 1e-12 * bn, &steps, &res)) return LB_CUDA_ERROR;
        inf.gmres_steps += steps;
        inf.refine_steps += 1;
        if (vec_axpby(wt, dw, nn, cmake(1, 0), cmake(1, 0), s)) return LB_CUDA_ERROR;
        if (change_basis(h, s, wt, w, h->X[2], 0)) return LB_CUDA_ERROR;
    }
    if (adjoint_residual(h, s, w, O, o.eta, R, &rmax, &rfro)) return LB_CUDA_ERROR;
    inf.residual_max = rmax;
    inf.residual_fro = rfro;
    // sensitivity matrices
    cplx* Ws = h->X[5];
    cplx* Rs = h->X[6];
    cplx* t1 = h->X[7];
    if (gH_dev) {
        cplx* gH = (cplx*)gH_dev;
        // G_H = i (rho w - w rho)
        if (gemm(h, s, gH, rho, OP_N, w, OP_N, n, n, n, cmake(0, 1), cmake(0, 0))) return LB_CUDA_ERROR;
        if (gemm(h, s, gH, w, OP_N, rho, OP_N, n, n, n, cmake(0, -1), cmake(1, 0))) return LB_CUDA_ERROR;
    }
    if (gL_dev) {
        cplx* gL = (cplx*)gL_dev;
        k_herm_sum<<<grid1(nn), 256, 0, s>>>(Ws, w, n); lb_note_launch();
        // Rs = Ws rho + rho Ws
        if (gemm(h, s, Rs, Ws, OP_N, rho, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return LB_CUDA_ERROR;
        if (gemm(h, s, Rs, rho, OP_N, Ws, OP_N, n, n, n, cmake(1, 0), cmake(1, 0))) return LB_CUDA_ERROR;
        for (int j = 0; j < d; ++j) {
            const cplx* Lj = h->L + (size_t)j * nn;
            cplx* gj = gL + (size_t)j * nn;
            // G_L_j = 1/2 L_j Rs - (Ws L_j) rho
            if (gemm(h, s, t1, Ws, OP_N, Lj, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return LB_CUDA_ERROR;
            if (gemm(h, s, gj, Lj, OP_N, Rs, OP_N, n, n, n, cmake(0.5, 0), cmake(0, 0))) return LB_CUDA_ERROR;
            if (gemm(h, s, gj, t1, OP_N, rho, OP_N, n, n, n, cmake(-1, 0), cmake(1, 0))) return LB_CUDA_ERROR;
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return LB_CUDA_ERROR;
    st = rmax < o.tol ? LB_OK : LB_NOT_CONVERGED;
    inf.status = st;
    if (info) *info = inf;
    return st;
}

extern "C" lb_status steady_state_adjoint(lindblad_handle h, const void* rho_dev, const void* O_dev, void* w_dev,
                                          void* gH_dev, void* gL_dev, const lb_opts* opts, lb_info* info,
                                          void* stream) {
    return device_error_guard(h, (cudaStream_t)stream, steady_state_adjoint_body(h, rho_dev, O_dev, w_dev, gH_dev, gL_dev, opts, info, stream));
}
