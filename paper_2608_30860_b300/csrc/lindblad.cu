// C ABI of the Lindblad library: set-up, Phi / resolvent / Lindbladian application and the
// host-side sequencing of the Krylov solvers (Alg. 4 steady state, Alg. 5 low spectrum).
// The host only sequences launches and reads back the per-restart stopping quantities;
// every arithmetic step on matrices runs in the kernels of this directory.
#include <cusolverDn.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <set>
#include <tuple>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/lindblad.h"
#include "common.cuh"
#include "lb_internal.cuh"
#include "vecops.cuh"

// ============================================================================ workspace layout
namespace {

struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

int krylov_cap(const lb_opts* o) {
    int m = o ? o->krylov_m : 20;
    int g = o ? o->gmres_m : 40;
    return std::max(std::max(m, g), 4);
}

// recycled-GMRES capacity: opts->recycle_k clipped to [0, 16] and to gmres_m - 2
int recycle_cap(const lb_opts* o) {
    int k = o ? o->recycle_k : 8;
    int g = o ? o->gmres_m : 40;
    return std::max(0, std::min(std::min(k, 16), g - 2));
}

size_t cusolver_ws_bytes(int n, size_t* host_bytes) {
    cusolverDnHandle_t hs = nullptr;
    cusolverDnParams_t prm = nullptr;
    size_t dev_geev = 0, host_geev = 0, dev_qr = 0, host_qr = 0;
    int lwork = 0;
    if (cusolverDnCreate(&hs) != CUSOLVER_STATUS_SUCCESS) return 0;
    cusolverDnCreateParams(&prm);
    cusolverDnXgeev_bufferSize(hs, prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, CUDA_C_64F,
                               nullptr, n, CUDA_C_64F, nullptr, CUDA_C_64F, nullptr, n, CUDA_C_64F, nullptr, n,
                               CUDA_C_64F, &dev_geev, &host_geev);
    cusolverDnXgeqrf_bufferSize(hs, prm, n, n, CUDA_C_64F, nullptr, n, CUDA_C_64F, nullptr, CUDA_C_64F, &dev_qr,
                                &host_qr);
    cusolverDnZungqr_bufferSize(hs, n, n, n, nullptr, n, nullptr, &lwork);
    size_t dev_tri = 0, host_tri = 0;
    cusolverDnXtrtri_bufferSize(hs, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, n, CUDA_C_64F, nullptr, n, &dev_tri,
                                &host_tri);
    dev_qr = std::max(dev_qr, dev_tri);
    host_qr = std::max(host_qr, host_tri);
    cusolverDnDestroyParams(prm);
    cusolverDnDestroy(hs);
    if (host_bytes) *host_bytes = std::max(host_geev, host_qr);
    size_t ung = (size_t)lwork * sizeof(cplx);
    return std::max(std::max(dev_geev, dev_qr), ung) + 4096;
}

// Lays out every device buffer of a handle; with base == nullptr only counts bytes.
void layout(lb_handle_s* h, char* base, int n, int d, const lb_opts* o, size_t solver_ws) {
    Carver c{base};
    const size_t nn = (size_t)n * n;
    h->H = c.take<cplx>(nn);
    h->L = c.take<cplx>((size_t)d * nn);
    h->G = c.take<cplx>(nn);
    h->Q = c.take<cplx>(nn);
    h->T = c.take<cplx>(nn);
    h->Lt = c.take<cplx>((size_t)d * nn);
    h->P = c.take<cplx>(std::max((size_t)d * nn, mixed_P_rows(n, d) * (size_t)n));
    for (int i = 0; i < NSCRATCH; ++i) h->X[i] = c.take<cplx>(nn);
    h->best = c.take<cplx>(nn);
    h->Rres = c.take<cplx>(nn);
    h->bk0 = c.take<cplx>(nn);
    h->bk1 = c.take<cplx>(nn);
    h->W = c.take<cplx>(nn);
    h->Wa = c.take<cplx>(nn);
    h->Ua = c.take<cplx>(nn);
    h->Re = c.take<cplx>(nn);
    h->Rinv = c.take<cplx>(nn);
    h->E1 = c.take<cplx>(nn);
    h->E2 = c.take<cplx>(nn);
    h->vcap = krylov_cap(o) + 1;
    h->V = c.take<cplx>((size_t)h->vcap * nn);
    h->Z = c.take<cplx>((size_t)h->vcap * nn);
    h->ldh = KMAX + 1;
    h->hm = c.take<cplx>((size_t)(KMAX + 1) * (KMAX + 1));
    h->hm2 = c.take<cplx>((size_t)(KMAX + 1) * (KMAX + 1));
    h->ev = c.take<cplx>(KMAX + 2);
    h->evec = c.take<cplx>((size_t)(KMAX + 2) * (KMAX + 2));
    h->small = c.take<cplx>(4 * (KMAX + 2));
    h->part = c.take<cplx>((size_t)DOT_BLOCKS * (KMAX + 2));
    h->dpart = c.take<double>(2 * DOT_BLOCKS);
    h->dscal = c.take<double>(16);
    h->scal = c.take<cplx>(16);
    h->dinfo = c.take<int>(16);
    h->solver_ws = c.take<char>(solver_ws);
    h->solver_ws_bytes = solver_ws;
    h->mixed_base = c.take<char>(mixed_bytes(n, d));
    {
        const int rk = recycle_cap(o);
        h->n = n;
        char* rb = c.take<char>(recycle_bytes(n, rk));
        if (base) recycle_layout(h, rb, rk);
        h->rk = rk;
    }
    h->ws_bytes = c.off + 256;
}

}  // namespace

// ============================================================================ launch counter
static std::atomic<long long> g_launches{0};
void lb_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// cudaFuncSetAttribute applies per device: remember (kernel, device, bytes) pairs already raised
int lb_smem_attr(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::set<std::tuple<const void*, int, int>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(kernel, dev, bytes);
    if (done.count(key)) return 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return -1;
    done.insert(key);
    return 0;
}

// ============================================================================ kernel timing
void prof_begin(lb_handle_s* h, cudaStream_t s, int kid) {
    if (!h->profiling) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    h->prof_ev[kid].push_back(e);
}
void prof_end(lb_handle_s* h, cudaStream_t s, int kid, double flops) {
    if (!h->profiling) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    h->prof_ev[kid].push_back(e);
    h->prof_flops[kid].push_back(flops);
}
static void prof_clear(lb_handle_s* h) {
    for (int k = 0; k < 2; ++k) {
        for (cudaEvent_t e : h->prof_ev[k]) cudaEventDestroy(e);
        h->prof_ev[k].clear();
        h->prof_flops[k].clear();
    }
}

// ============================================================================ GEMM shorthands
int gemm(lb_handle_s* h, cudaStream_t s, cplx* C, const cplx* A, int opA, const cplx* B, int opB, int M, int N,
         int K, cplx alpha, cplx beta) {
    ZGemmArgs a{};
    a.M = M; a.N = N; a.K = K;
    a.A = A; a.lda = (opA == OP_N) ? K : M; a.strideA = 0; a.opA = opA;
    a.B = B; a.ldb = (opB == OP_N) ? N : K; a.strideB = 0; a.opB = opB;
    a.C = C; a.ldc = N; a.strideC = 0;
    a.alpha = alpha; a.beta = beta; a.batch = 1; a.reduce = 1;
    prof_begin(h, s, 1);
    int r = zgemm_f64(a, s);
    prof_end(h, s, 1, 8.0 * M * (double)N * K);
    return r;
}

// Y = alpha * sum_j Lop_j Z Lop_j^dag + beta Y, with Lop the stack Ls (d x n x n), in FP64.  herm = 1
// (Z Hermitian, alpha and beta real, Y Hermitian on entry): the second product is Hermitian, so only
// its upper tiles are computed and the rest mirrored.
int jump_f64(lb_handle_s* h, cudaStream_t s, const cplx* Ls, const cplx* Z, cplx* Y, cplx alpha, cplx beta, int herm) {
    const int n = h->n, d = h->d;
    const long long nn = (long long)n * n;
    // P = [L_1; ...; L_d] Z  (dn x n)
    if (gemm(h, s, h->P, Ls, OP_N, Z, OP_N, d * n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    // Y = alpha sum_j P_j L_j^dag + beta Y
    ZGemmArgs a{};
    a.M = n; a.N = n; a.K = n;
    a.A = h->P; a.lda = n; a.strideA = nn; a.opA = OP_N;
    a.B = Ls; a.ldb = n; a.strideB = nn; a.opB = OP_C;
    a.C = Y; a.ldc = n; a.strideC = 0;
    a.alpha = alpha; a.beta = beta; a.batch = d; a.reduce = 1; a.herm = herm;
    prof_begin(h, s, 1);
    int r = zgemm_f64(a, s);
    prof_end(h, s, 1, (herm ? 4.0 * (n + 1) : 8.0 * n) * (double)n * n * d);
    return r;
}

// R = L(X) = G X + X G^dag + sum_j L_j X L_j^dag, FP64, original basis
int lindbladian_f64(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* R) {
    const int n = h->n;
    if (gemm(h, s, R, h->G, OP_N, X, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    if (gemm(h, s, R, X, OP_N, h->G, OP_C, n, n, n, cmake(1, 0), cmake(1, 0))) return -1;
    return jump_f64(h, s, h->L, X, R, cmake(1, 0), cmake(1, 0));
}

// the same for Hermitian X: X G^dag = (G X)^dag, so one GEMM and an adjoint-add form the no-jump part,
// and the jump part is Hermitian (upper tiles only)
int lindbladian_f64_herm(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* R) {
    const int n = h->n;
    if (gemm(h, s, R, h->G, OP_N, X, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    if (mat_add_adjoint(R, n, s)) return -1;
    return jump_f64(h, s, h->L, X, R, cmake(1, 0), cmake(1, 0), 1);
}

// Out = Q X Q^dag (to_schur = 0) or Q^dag X Q (to_schur = 1); tmp must differ from X and Out
int change_basis(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* Out, cplx* tmp, int to_schur) {
    const int n = h->n;
    if (to_schur) {
        if (gemm(h, s, tmp, h->Q, OP_C, X, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
        return gemm(h, s, Out, tmp, OP_N, h->Q, OP_N, n, n, n, cmake(1, 0), cmake(0, 0));
    }
    if (gemm(h, s, tmp, h->Q, OP_N, X, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    return gemm(h, s, Out, tmp, OP_N, h->Q, OP_C, n, n, n, cmake(1, 0), cmake(0, 0));
}

// Schur-coordinate Lyapunov solve: X solves (T - s I) X + X (T - s I)^dag = Y (X may equal Y)
int lyap_schur(lb_handle_s* h, cudaStream_t s, const cplx* Y, cplx* X, double shift, int precision) {
    const long long nn = (long long)h->n * h->n;
    if (X != Y) LB_CHECK_CUDA(cudaMemcpyAsync(X, Y, nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    if (precision == LB_PREC_MIXED && h->mixed_sylv_ready) return trisylv_mixed(h, s, X, shift);
    if (h->eig_active) return lyap_eig(h, s, X, X, shift);
    return trisylv_f64(h->T, X, h->n, cmake(shift, 0.0), s);
}

// eigenbasis route (Alg. 1) in Schur coordinates: X = R[(R^{-1} Y R^{-dag}) o D]R^dag,
// D_ij = 1 / (s_i + conj(s_j) - 2 shift), s = diag(T); Y and X may alias
int lyap_eig(lb_handle_s* h, cudaStream_t s, const cplx* Y, cplx* X, double shift) {
    const int n = h->n;
    cplx* t = h->E1;
    cplx* yh = h->E2;
    if (gemm(h, s, t, h->Rinv, OP_N, Y, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    if (gemm(h, s, yh, t, OP_N, h->Rinv, OP_C, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    if (mat_eig_divide(yh, h->T, n, shift, s)) return -1;
    if (gemm(h, s, t, h->Re, OP_N, yh, OP_N, n, n, n, cmake(1, 0), cmake(0, 0))) return -1;
    return gemm(h, s, X, t, OP_N, h->Re, OP_C, n, n, n, cmake(1, 0), cmake(0, 0));
}

// Schur-coordinate Phi (form 0) or M (form 1): Y = -K~ S~^{-1} X  or  Y = -S~^{-1} K~ X.  herm = 1: X is
// Hermitian, so is every intermediate (S~^{-1} and K~ preserve Hermiticity) and the jump term's second
// product is formed on its upper tiles only.
int phi_schur(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* Y, int form, int precision, int herm) {
    cplx* Z = h->X[0];
    const long long nn = (long long)h->n * h->n;
    if (form == 0) {
        if (lyap_schur(h, s, X, Z, 0.0, precision)) return -1;
        if (precision == LB_PREC_MIXED && h->mixed_ready) return jump_mixed(h, s, Z, Y, -1.0, herm);
        return jump_f64(h, s, h->Lt, Z, Y, cmake(-1, 0), cmake(0, 0), herm);
    }
    if (precision == LB_PREC_MIXED && h->mixed_ready) {
        if (jump_mixed(h, s, X, Z, 1.0, herm)) return -1;
    } else if (jump_f64(h, s, h->Lt, X, Z, cmake(1, 0), cmake(0, 0), herm)) {
        return -1;
    }
    if (lyap_schur(h, s, Z, Z, 0.0, precision)) return -1;
    return vec_scale_copy(Y, Z, nn, cmake(-1, 0), s);
}

// ============================================================================ Arnoldi
// One Arnoldi cycle of length up to m on op, starting from V[0] (unit norm).  Classical
// Gram-Schmidt applied twice per step; the Hessenberg column lives on the device
// (column-major, leading dimension ldh).  Breakdown is detected on the device (the step is
// recorded and the later basis vectors are zero), so the host synchronises once per cycle, not
// once per step.  Returns the number of completed steps in *k_out.
int arnoldi_cycle(lb_handle_s* h, cudaStream_t s, cplx* basis, cplx* hess, int j0, int m, const OpFn& op,
                  int* k_out) {
    const long long nn = (long long)h->n * h->n;
    cplx* hc2 = h->small;
    cplx* nrm2 = h->small + (KMAX + 2);
    cplx* inv = h->small + 2 * (KMAX + 2);
    // one flag per nesting level: the shift-invert Arnoldi runs an inner GMRES cycle inside each step
    if (h->arn_depth >= 4) return -1;
    int* brk = h->dinfo + 12 + h->arn_depth;
    struct Depth {
        int& d;
        explicit Depth(int& v) : d(v) { ++d; }
        ~Depth() { --d; }
    } depth_guard(h->arn_depth);
    LB_CHECK_CUDA(cudaMemsetAsync(brk, 0, sizeof(int), s));
    for (int k = j0; k < m; ++k) {
        cplx* w = basis + (k + 1) * nn;
        cplx* hcol = hess + (size_t)k * h->ldh;
        if (op(basis + k * nn, w)) return -1;
        for (int pass = 0; pass < 2; ++pass) {
            cplx* out = pass == 0 ? hcol : hc2;
            if (vec_dot_block(basis, nn, k + 1, w, nn, out, h->part, 0, s)) return -1;
            if (vec_gemv(w, basis, nn, k + 1, out, nn, -1.0, 1, s)) return -1;
        }
        if (vec_dot_block(w, nn, 1, w, nn, nrm2, h->part, 0, s)) return -1;
        if (vec_finish_column(hcol, hc2, k + 1, nrm2, inv, s, brk)) return -1;
        if (vec_scale_dev(w, nn, inv, s)) return -1;
    }
    int kb = 0;
    LB_CHECK_CUDA(cudaMemcpyAsync(&kb, brk, sizeof(int), cudaMemcpyDeviceToHost, s));
    LB_CHECK_CUDA(cudaStreamSynchronize(s));
    *k_out = (kb > 0 && kb < m) ? kb : m;
    return 0;
}

// ============================================================================ helpers
namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// index of the Ritz value nearest 1; ties -> larger Re -> smaller index
int pick_nearest_one(const std::vector<std::complex<double>>& th) {
    int best = 0;
    for (int i = 1; i < (int)th.size(); ++i) {
        double di = std::abs(th[i] - 1.0), db = std::abs(th[best] - 1.0);
        if (di < db - 1e-15 || (std::fabs(di - db) <= 1e-15 && th[i].real() > th[best].real())) best = i;
    }
    return best;
}

}  // namespace

// (rho / Tr rho), hermitised, renormalised: in -> out (out may equal in); tmp scratch
int hermitize_normalize(lb_handle_s* h, cudaStream_t s, const cplx* in, cplx* out, cplx* tmp) {
    const int n = h->n;
    const long long nn = (long long)n * n;
    if (mat_trace(in, n, h->scal, s)) return -1;
    if (mat_div_by_dev(tmp, in, nn, h->scal, s)) return -1;
    if (mat_hermitize(out, tmp, n, s)) return -1;
    if (mat_trace(out, n, h->scal + 1, s)) return -1;
    return mat_div_by_dev(out, out, nn, h->scal + 1, s, 1);   // Hermitian: divide by the real trace
}

// max-norm and Frobenius norm of L(rho), rho in the original basis; R scratch
int residual_norms(lb_handle_s* h, cudaStream_t s, const cplx* rho, cplx* R, double* rmax, double* rfro) {
    // rho is Hermitian here (every caller hermitises first)
    if (lindbladian_f64_herm(h, s, rho, R)) return -1;
    if (vec_norms(R, (long long)h->n * h->n, h->dpart, h->dscal, s)) return -1;
    double out[2];
    LB_CHECK_CUDA(cudaMemcpyAsync(out, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LB_CHECK_CUDA(cudaStreamSynchronize(s));
    *rmax = out[0];
    *rfro = out[1];
    return 0;
}

// reads (and clears) the device error word set by bounded waits in the tensor-core kernels
lb_status check_device_error(lb_handle_s* h, cudaStream_t s) {
    int e = 0;
    LB_CHECK_CUDA(cudaMemcpyAsync(&e, h->dinfo + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
    LB_CHECK_CUDA(cudaStreamSynchronize(s));
    if (e != 0) {
        fprintf(stderr, "lindblad: tensor-core kernel wait timed out (code %d)\n", e);
        cudaMemsetAsync(h->dinfo + 8, 0, sizeof(int), s);
        return LB_CUDA_ERROR;
    }
    return LB_OK;
}

// the status of an entry point, or LB_CUDA_ERROR when a bounded wait of a tensor-core kernel gave up
// during the call (the result is then not valid); the error word is cleared
lb_status device_error_guard(lb_handle_s* h, cudaStream_t s, lb_status st) {
    if (!h) return st;
    const lb_status e = check_device_error(h, s);
    return e != LB_OK ? e : st;
}

// ============================================================================ C ABI
extern "C" {

void lb_default_opts(lb_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->krylov_m = 20;
    o->max_restarts = 60;
    o->precision = LB_PREC_FP64;
    o->eta = 1.0;
    o->max_refine = 8;
    o->gmres_m = 40;
    o->sylv_block = 0;
    o->inner_tol = 1e-10;
    o->keep_ritz = 0;
    o->route = LB_ROUTE_SCHUR;
    o->eig_cond_max = 1e3;
    o->schur_tol = 1e-12;
    o->recycle_k = 8;
    o->gauge_c = nullptr;
    o->batched_tiles = nullptr;
}

const char* lb_status_string(int st) {
    switch (st) {
        case LB_OK: return "LB_OK";
        case LB_NOT_CONVERGED: return "LB_NOT_CONVERGED";
        case LB_S_SINGULAR: return "LB_S_SINGULAR";
        case LB_ILL_CONDITIONED: return "LB_ILL_CONDITIONED";
        case LB_INVALID_ARG: return "LB_INVALID_ARG";
        case LB_CUDA_ERROR: return "LB_CUDA_ERROR";
        case LB_ETA_EXCLUDED: return "LB_ETA_EXCLUDED";
        case LB_WORKSPACE_TOO_SMALL: return "LB_WORKSPACE_TOO_SMALL";
        case LB_NOT_IMPLEMENTED: return "LB_NOT_IMPLEMENTED";
        case LB_SOLVER_ERROR: return "LB_SOLVER_ERROR";
        default: return "LB_UNKNOWN";
    }
}

size_t lindblad_workspace_bytes(int n, int d, const lb_opts* opts) {
    if (n < 2 || d < 1) return 0;
    lb_opts o;
    lb_default_opts(&o);
    if (opts) o = *opts;
    if (krylov_cap(&o) > KMAX) return 0;
    lb_handle_s tmp{};
    size_t host = 0;
    size_t sws = cusolver_ws_bytes(n, &host);
    if (sws == 0) return 0;
    layout(&tmp, nullptr, n, d, &o, sws);
    return tmp.ws_bytes;
}

lb_status lindblad_setup(const void* H_dev, const void* L_dev, int n, int d, void* workspace, size_t ws_bytes,
                         void* stream, const lb_opts* opts, lindblad_handle* out, lb_info* info) {
    if (!H_dev || !L_dev || !workspace || !out || n < 2 || d < 1) return LB_INVALID_ARG;
    lb_opts o;
    lb_default_opts(&o);
    if (opts) o = *opts;
    if (krylov_cap(&o) > KMAX || o.krylov_m < 2) return LB_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = now_ms();
    size_t host_bytes = 0;
    size_t sws = cusolver_ws_bytes(n, &host_bytes);
    if (sws == 0) return LB_SOLVER_ERROR;
    lb_handle_s* h = new lb_handle_s{};
    h->n = n;
    h->d = d;
    h->opts = o;
    layout(h, nullptr, n, d, &o, sws);
    if (h->ws_bytes > ws_bytes) { delete h; return LB_WORKSPACE_TOO_SMALL; }
    layout(h, (char*)workspace, n, d, &o, sws);
    const long long nn = (long long)n * n;
    auto fail = [&](lb_status st) { delete h; return st; };

    if (cudaMemcpyAsync(h->H, H_dev, nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->L, L_dev, (size_t)d * nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(LB_CUDA_ERROR);
    {
        // NaN or Inf in H or L_j: refused before any factorisation (the sum of squares of the entries is
        // finite exactly when every entry is finite and below ~1e154)
        double fro[2] = {0.0, 0.0};
        if (vec_norms(h->H, nn, h->dpart, h->dscal, s)) return fail(LB_CUDA_ERROR);
        if (cudaMemcpyAsync(&fro[0], h->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return fail(LB_CUDA_ERROR);
        if (vec_norms(h->L, (long long)d * nn, h->dpart, h->dscal, s)) return fail(LB_CUDA_ERROR);
        if (cudaMemcpyAsync(&fro[1], h->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(LB_CUDA_ERROR);
        if (!std::isfinite(fro[0]) || !std::isfinite(fro[1])) return fail(LB_INVALID_ARG);
    }
    if (o.gauge_c) {
        // gauge of the split: the handle then holds (H~, L~_j); L is unchanged, S~ and K~ are not
        if (cudaMemcpyAsync(h->part, o.gauge_c, (size_t)d * sizeof(cplx), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            gauge_split(h->H, h->L, n, d, h->part, s))
            return fail(LB_CUDA_ERROR);
        h->gauged = true;
    }
    // G = -iH - 1/2 sum_j L_j^dag L_j: the sum is Hermitian, so one stacked GEMM (K = d n) on its upper
    // tiles plus the mirror, then the anti-Hermitian part -iH added
    {
        ZGemmArgs a{};
        a.M = n; a.N = n; a.K = d * n;
        a.A = h->L; a.lda = n; a.strideA = 0; a.opA = OP_C;
        a.B = h->L; a.ldb = n; a.strideB = 0; a.opB = OP_N;
        a.C = h->X[0]; a.ldc = n; a.strideC = 0;
        a.alpha = cmake(-0.5, 0); a.beta = cmake(0, 0); a.batch = 1; a.reduce = 1; a.herm = 1;
        if (zgemm_f64(a, s)) return fail(LB_CUDA_ERROR);
    }
    if (vec_scale_copy(h->G, h->H, nn, cmake(0, -1), s)) return fail(LB_CUDA_ERROR);
    if (vec_axpby(h->G, h->X[0], nn, cmake(1, 0), cmake(1, 0), s)) return fail(LB_CUDA_ERROR);
    // eigenvectors of G (column-major view of G^T storage is G), QR of them -> Schur vectors
    cplx* Acm = h->X[0];
    cplx* VR = h->X[1];
    cplx* W = h->X[2];   // eigenvalues (n entries)
    cplx* tau = h->X[3];
    if (mat_transpose(Acm, h->G, n, s)) return fail(LB_CUDA_ERROR);
    {
        cusolverDnHandle_t hs = nullptr;
        cusolverDnParams_t prm = nullptr;
        if (cusolverDnCreate(&hs) != CUSOLVER_STATUS_SUCCESS) return fail(LB_SOLVER_ERROR);
        cusolverDnSetStream(hs, s);
        cusolverDnCreateParams(&prm);
        std::vector<char> hbuf(std::max<size_t>(host_bytes, 16));
        size_t dws = 0, hws = 0;
        cusolverStatus_t cs = cusolverDnXgeev_bufferSize(
            hs, prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, CUDA_C_64F, Acm, n, CUDA_C_64F, W,
            CUDA_C_64F, nullptr, n, CUDA_C_64F, VR, n, CUDA_C_64F, &dws, &hws);
        if (hws > hbuf.size()) hbuf.resize(hws);
        if (cs == CUSOLVER_STATUS_SUCCESS && dws <= h->solver_ws_bytes)
            cs = cusolverDnXgeev(hs, prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, CUDA_C_64F, Acm,
                                 n, CUDA_C_64F, W, CUDA_C_64F, nullptr, n, CUDA_C_64F, VR, n, CUDA_C_64F,
                                 h->solver_ws, h->solver_ws_bytes, hbuf.data(), hbuf.size(), h->dinfo);
        else if (cs == CUSOLVER_STATUS_SUCCESS)
            cs = CUSOLVER_STATUS_ALLOC_FAILED;
        int dinfo = 0;
        if (cs == CUSOLVER_STATUS_SUCCESS) {
            cudaMemcpyAsync(&dinfo, h->dinfo, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
        }
        if (cs == CUSOLVER_STATUS_SUCCESS && dinfo == 0) {
            cs = cusolverDnXgeqrf_bufferSize(hs, prm, n, n, CUDA_C_64F, VR, n, CUDA_C_64F, tau, CUDA_C_64F, &dws,
                                             &hws);
            if (hws > hbuf.size()) hbuf.resize(hws);
            if (cs == CUSOLVER_STATUS_SUCCESS && dws > h->solver_ws_bytes) cs = CUSOLVER_STATUS_ALLOC_FAILED;
            if (cs == CUSOLVER_STATUS_SUCCESS)
                cs = cusolverDnXgeqrf(hs, prm, n, n, CUDA_C_64F, VR, n, CUDA_C_64F, tau, CUDA_C_64F, h->solver_ws,
                                      h->solver_ws_bytes, hbuf.data(), hbuf.size(), h->dinfo);
            // eigenbasis route: R = Q^dag U is the triangular QR factor held in VR's upper triangle
            if (cs == CUSOLVER_STATUS_SUCCESS && o.route != LB_ROUTE_SCHUR) {
                cplx* Rcm = h->X[4];
                if (mat_transpose(h->X[5], VR, n, s) || mat_take_upper(h->Re, h->X[5], n, h->dpart, h->dscal + 6, s) ||
                    cudaMemcpyAsync(Rcm, VR, (size_t)nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    cs = CUSOLVER_STATUS_EXECUTION_FAILED;
                size_t dt = 0, ht = 0;
                if (cs == CUSOLVER_STATUS_SUCCESS)
                    cs = cusolverDnXtrtri_bufferSize(hs, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, n, CUDA_C_64F,
                                                     Rcm, n, &dt, &ht);
                if (ht > hbuf.size()) hbuf.resize(ht);
                if (cs == CUSOLVER_STATUS_SUCCESS && dt > h->solver_ws_bytes) cs = CUSOLVER_STATUS_ALLOC_FAILED;
                if (cs == CUSOLVER_STATUS_SUCCESS)
                    cs = cusolverDnXtrtri(hs, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, n, CUDA_C_64F, Rcm, n,
                                          h->solver_ws, h->solver_ws_bytes, hbuf.data(), hbuf.size(), h->dinfo);
                if (cs == CUSOLVER_STATUS_SUCCESS &&
                    (mat_transpose(h->X[5], Rcm, n, s) || mat_take_upper(h->Rinv, h->X[5], n, h->dpart, h->dscal + 6, s)))
                    cs = CUSOLVER_STATUS_EXECUTION_FAILED;
            }
            int lwork = 0;
            if (cs == CUSOLVER_STATUS_SUCCESS)
                cs = cusolverDnZungqr_bufferSize(hs, n, n, n, (cuDoubleComplex*)VR, n, (cuDoubleComplex*)tau, &lwork);
            if (cs == CUSOLVER_STATUS_SUCCESS && (size_t)lwork * sizeof(cplx) > h->solver_ws_bytes)
                cs = CUSOLVER_STATUS_ALLOC_FAILED;
            if (cs == CUSOLVER_STATUS_SUCCESS)
                cs = cusolverDnZungqr(hs, n, n, n, (cuDoubleComplex*)VR, n, (cuDoubleComplex*)tau,
                                      (cuDoubleComplex*)h->solver_ws, lwork, h->dinfo);
            if (cs == CUSOLVER_STATUS_SUCCESS) {
                cudaMemcpyAsync(&dinfo, h->dinfo, sizeof(int), cudaMemcpyDeviceToHost, s);
                cudaStreamSynchronize(s);
            }
        }
        cusolverDnDestroyParams(prm);
        cusolverDnDestroy(hs);
        if (cs != CUSOLVER_STATUS_SUCCESS || dinfo != 0) {
            fprintf(stderr, "lindblad: cusolver status %d info %d in set-up\n", (int)cs, dinfo);
            return fail(LB_SOLVER_ERROR);
        }
    }
    // Q (row-major) = transpose of the column-major Schur-vector array
    if (mat_transpose(h->Q, VR, n, s)) return fail(LB_CUDA_ERROR);
    // A = Q^dag G Q ; T = upper(A) ; backward error = ||lower(A)||_F / ||G||_F
    if (change_basis(h, s, h->G, h->X[1], h->X[0], 1)) return fail(LB_CUDA_ERROR);
    if (mat_take_upper(h->T, h->X[1], n, h->dpart, h->dscal, s)) return fail(LB_CUDA_ERROR);
    if (vec_norms(h->G, nn, h->dpart, h->dscal + 2, s)) return fail(LB_CUDA_ERROR);
    if (mat_min_abs_re_diag(h->T, n, h->dscal + 4, s)) return fail(LB_CUDA_ERROR);
    // L~_j = Q^dag L_j Q (batched)
    {
        ZGemmArgs a{};
        a.M = n; a.N = n; a.K = n;
        a.A = h->Q; a.lda = n; a.strideA = 0; a.opA = OP_C;
        a.B = h->L; a.ldb = n; a.strideB = nn; a.opB = OP_N;
        a.C = h->P; a.ldc = n; a.strideC = nn;
        a.alpha = cmake(1, 0); a.beta = cmake(0, 0); a.batch = d; a.reduce = 0;
        if (zgemm_f64(a, s)) return fail(LB_CUDA_ERROR);
        a.A = h->P; a.strideA = nn; a.opA = OP_N;
        a.B = h->Q; a.strideB = 0; a.opB = OP_N;
        a.C = h->Lt; a.strideC = nn;
        if (zgemm_f64(a, s)) return fail(LB_CUDA_ERROR);
    }
    double diag[6];
    if (cudaMemcpyAsync(diag, h->dscal, 6 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(LB_CUDA_ERROR);
    h->gnorm = diag[3];
    h->schur_err = diag[1] / std::max(diag[3], 1e-300);
    h->min_re_T = diag[4];
    h->case1 = h->min_re_T <= 1e3 * 2.220446049250313e-16 * h->gnorm;
    if (!(h->schur_err <= o.schur_tol)) {
        // the QR of the eigenvector matrix is not a backward-stable Schur form when the eigenvectors
        // are ill-conditioned: refuse rather than precondition with the factor of another matrix
        fprintf(stderr, "lindblad: Schur backward error %.3e above the gate %.3e\n", h->schur_err, o.schur_tol);
        if (info) {
            std::memset(info, 0, sizeof(*info));
            info->schur_backward_err = h->schur_err;
            info->min_abs_re_T = h->min_re_T;
            info->status = LB_SOLVER_ERROR;
        }
        return fail(LB_SOLVER_ERROR);
    }
    lb_status ret = LB_OK;
    if (o.route != LB_ROUTE_SCHUR) {
        double nr[4];
        if (vec_norms(h->Re, nn, h->dpart, h->dscal + 8, s) || vec_norms(h->Rinv, nn, h->dpart, h->dscal + 10, s) ||
            cudaMemcpyAsync(nr, h->dscal + 8, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(LB_CUDA_ERROR);
        h->cond_eig = nr[1] * nr[3] / n;
        h->eig_active = !h->case1 && std::isfinite(h->cond_eig) && h->cond_eig <= o.eig_cond_max;
        if (o.route == LB_ROUTE_EIG && !h->eig_active) ret = LB_ILL_CONDITIONED;
    }
    if (cudaMemsetAsync(h->dinfo, 0, 16 * sizeof(int), s) != cudaSuccess) return fail(LB_CUDA_ERROR);
    if (mixed_prepare(h, s)) return fail(LB_CUDA_ERROR);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(LB_CUDA_ERROR);
    h->setup_ms = now_ms() - t0;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->schur_backward_err = h->schur_err;
        info->min_abs_re_T = h->min_re_T;
        info->setup_ms = h->setup_ms;
        info->cond_eig = h->cond_eig;
        info->route = h->eig_active ? LB_ROUTE_EIG : LB_ROUTE_SCHUR;
        info->status = h->case1 ? LB_S_SINGULAR : ret;
    }
    *out = h;
    return ret;
}

void lindblad_destroy(lindblad_handle h) {
    if (h) prof_clear(h);
    delete h;
}

long long lb_launch_count(void) { return g_launches.load(); }

lb_status lb_set_profiling(lindblad_handle h, int enable) {
    if (!h) return LB_INVALID_ARG;
    prof_clear(h);
    h->profiling = enable != 0;
    return LB_OK;
}

lb_status lb_test_bounded_wait(lindblad_handle h, int stall_iteration, double wait_ms) {
    if (!h || !(wait_ms >= 0.0 && wait_ms <= 2000.0) || stall_iteration < -1) return LB_INVALID_ARG;
    h->tc_wait_ns = (unsigned long long)(wait_ms * 1e6);
    h->tc_stall = stall_iteration + 1;
    return LB_OK;
}

lb_status lb_kernel_stats(lindblad_handle h, int kernel, int* launches, double* total_ms, double* flops) {
    if (!h || kernel < 0 || kernel > 1) return LB_INVALID_ARG;
    const auto& ev = h->prof_ev[kernel];
    double ms = 0.0, fl = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
        LB_CHECK_CUDA(cudaEventSynchronize(ev[i + 1]));
        float t = 0.f;
        LB_CHECK_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        ms += t;
    }
    for (double f : h->prof_flops[kernel]) fl += f;
    if (launches) *launches = (int)(ev.size() / 2);
    if (total_ms) *total_ms = ms;
    if (flops) *flops = fl;
    return LB_OK;
}


lb_status phi_apply(lindblad_handle h, const void* X_dev, void* Y_dev, int flags, int precision, void* stream) {
    if (!h || !X_dev || !Y_dev || X_dev == Y_dev) return LB_INVALID_ARG;
    if (h->case1) return LB_S_SINGULAR;
    cudaStream_t s = (cudaStream_t)stream;
    const int form = flags & LB_APPLY_FORM_M ? 1 : 0;
    const int herm = flags & LB_APPLY_HERMITIAN ? 2 : 0;   // 2: an exactly Hermitian result (real diagonal)
    const cplx* X = (const cplx*)X_dev;
    cplx* Y = (cplx*)Y_dev;
    if (precision == LB_PREC_MIXED && !h->mixed_ready) return LB_NOT_IMPLEMENTED;
    if (flags & LB_APPLY_SCHUR) {
        if (phi_schur(h, s, X, Y, form, precision, herm)) return LB_CUDA_ERROR;
    } else {
        if (change_basis(h, s, X, h->X[1], h->X[2], 1)) return LB_CUDA_ERROR;
        if (phi_schur(h, s, h->X[1], h->X[3], form, precision, herm)) return LB_CUDA_ERROR;
        if (change_basis(h, s, h->X[3], Y, h->X[2], 0)) return LB_CUDA_ERROR;
    }
    return precision == LB_PREC_MIXED ? check_device_error(h, s) : LB_OK;
}

lb_status jump_apply(lindblad_handle h, const void* X_dev, void* Y_dev, int flags, int precision, void* stream) {
    if (!h || !X_dev || !Y_dev || X_dev == Y_dev) return LB_INVALID_ARG;
    if (precision == LB_PREC_MIXED && !h->mixed_ready) return LB_NOT_IMPLEMENTED;
    cudaStream_t s = (cudaStream_t)stream;
    const cplx* X = (const cplx*)X_dev;
    cplx* Y = (cplx*)Y_dev;
    const int herm = flags & LB_APPLY_HERMITIAN ? 2 : 0;   // 2: an exactly Hermitian result (real diagonal)
    if (!(flags & LB_APPLY_SCHUR)) {
        // original basis: L_j themselves (FP64), or via Schur coordinates on the tensor cores
        if (precision != LB_PREC_MIXED)
            return jump_f64(h, s, h->L, X, Y, cmake(1, 0), cmake(0, 0), herm) ? LB_CUDA_ERROR : LB_OK;
        if (change_basis(h, s, X, h->X[1], h->X[2], 1)) return LB_CUDA_ERROR;
        if (jump_mixed(h, s, h->X[1], h->X[3], 1.0, herm)) return LB_CUDA_ERROR;
        if (change_basis(h, s, h->X[3], Y, h->X[2], 0)) return LB_CUDA_ERROR;
        return check_device_error(h, s);
    }
    if (precision == LB_PREC_MIXED) {
        if (jump_mixed(h, s, X, Y, 1.0, herm)) return LB_CUDA_ERROR;
        return check_device_error(h, s);
    }
    return jump_f64(h, s, h->Lt, X, Y, cmake(1, 0), cmake(0, 0), herm) ? LB_CUDA_ERROR : LB_OK;
}

static lb_status resolvent_apply_body(lindblad_handle h, const void* Y_dev, void* X_dev, double lam, int precision,
                          void* stream) {
    if (!h || !Y_dev || !X_dev) return LB_INVALID_ARG;
    if (h->case1 && !(lam > 0.0)) return LB_S_SINGULAR;
    if (precision == LB_PREC_MIXED && !h->mixed_ready) return LB_NOT_IMPLEMENTED;
    cudaStream_t s = (cudaStream_t)stream;
    const long long nn = (long long)h->n * h->n;
    // (lam - S) X = Y  <=>  T_lam X~ + X~ T_lam^dag = -Q^dag Y Q,  T_lam = T - lam/2
    if (change_basis(h, s, (const cplx*)Y_dev, h->X[1], h->X[2], 1)) return LB_CUDA_ERROR;
    if (vec_scale_copy(h->X[1], h->X[1], nn, cmake(-1, 0), s)) return LB_CUDA_ERROR;
    if (lyap_schur(h, s, h->X[1], h->X[1], 0.5 * lam, precision)) return LB_CUDA_ERROR;
    if (change_basis(h, s, h->X[1], (cplx*)X_dev, h->X[2], 0)) return LB_CUDA_ERROR;
    return LB_OK;
}

lb_status resolvent_apply(lindblad_handle h, const void* Y_dev, void* X_dev, double lam, int precision,
                          void* stream) {
    return device_error_guard(h, (cudaStream_t)stream, resolvent_apply_body(h, Y_dev, X_dev, lam, precision, stream));
}

lb_status lindbladian_apply(lindblad_handle h, const void* X_dev, void* R_dev, void* stream) {
    if (!h || !X_dev || !R_dev || X_dev == R_dev) return LB_INVALID_ARG;
    return lindbladian_f64(h, (cudaStream_t)stream, (const cplx*)X_dev, (cplx*)R_dev) ? LB_CUDA_ERROR : LB_OK;
}

static lb_status steady_state_body(lindblad_handle h, void* rho_dev, const lb_opts* opts, lb_info* info, void* stream) {
    if (!h || !rho_dev) return LB_INVALID_ARG;
    lb_opts o = h->opts;
    if (opts) o = *opts;
    if (o.krylov_m < 2 || o.krylov_m + 1 > h->vcap || o.krylov_m > KMAX) return LB_INVALID_ARG;
    if (o.precision == LB_PREC_MIXED && !h->mixed_ready) return LB_NOT_IMPLEMENTED;
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = now_ms();
    lb_info inf{};
    inf.schur_backward_err = h->schur_err;
    inf.min_abs_re_T = h->min_re_T;
    inf.setup_ms = h->setup_ms;
    inf.cond_eig = h->cond_eig;
    inf.route = h->eig_active && o.precision == LB_PREC_FP64 ? LB_ROUTE_EIG : LB_ROUTE_SCHUR;
    lb_status st = LB_OK;
    if (h->case1) {
        // Theorem 1, case 1: pure steady state from the eigenvector of G on the imaginary axis
        if (pure_state_case1(h, s, (cplx*)rho_dev)) return LB_CUDA_ERROR;
        double rmax, rfro;
        if (residual_norms(h, s, (cplx*)rho_dev, h->X[0], &rmax, &rfro)) return LB_CUDA_ERROR;
        inf.residual_max = rmax;
        inf.residual_fro = rfro;
        st = LB_S_SINGULAR;
    } else {
        st = steady_state_arnoldi(h, s, o, (cplx*)rho_dev, &inf);
        if (st >= 0 && o.precision == LB_PREC_MIXED && inf.residual_max >= o.tol) {
            st = refine_steady_state(h, s, o, (cplx*)rho_dev, &inf);
        }
    }
    inf.status = st;
    inf.solve_ms = now_ms() - t0;
    if (info) *info = inf;
    return st;
}

lb_status steady_state(lindblad_handle h, void* rho_dev, const lb_opts* opts, lb_info* info, void* stream) {
    return device_error_guard(h, (cudaStream_t)stream, steady_state_body(h, rho_dev, opts, info, stream));
}

}  // extern "C"

// ============================================================================ Alg. 4
lb_status steady_state_arnoldi(lb_handle_s* h, cudaStream_t s, const lb_opts& o, cplx* rho_out, lb_info* inf) {
    const int n = h->n;
    const long long nn = (long long)n * n;
    const int m = o.krylov_m;
    const int prec = o.precision;
    cplx* xi = h->X[2];
    cplx* rt = h->X[3];     // rho in Schur coordinates
    cplx* rho = h->X[4];    // rho in the original basis
    cplx* R = h->X[5];
    double best = INFINITY;
    // start vector I/n, normalised: I/sqrt(n)  (Schur-coordinate invariant)
    if (mat_eye(h->V, n, cmake(1.0 / std::sqrt((double)n), 0.0), s)) return LB_CUDA_ERROR;
    // the Krylov vectors of Phi from the Hermitian start I/sqrt(n) are Hermitian (real Hessenberg)
    OpFn op = [&](const cplx* x, cplx* y) { return phi_schur(h, s, x, y, 0, prec, 1); };
    std::vector<cplx> evh(KMAX);
    double prev_ritz = INFINITY;
    int restart = 0;
    for (; restart < o.max_restarts; ++restart) {
        int k = 0;
        if (arnoldi_cycle(h, s, h->V, h->hm, 0, m, op, &k)) return LB_CUDA_ERROR;
        inf->phi_applies += k;
        if (hess_eig(h->hm, h->ldh, k, h->ev, h->evec, h->dinfo, s)) return LB_CUDA_ERROR;
        LB_CHECK_CUDA(cudaMemcpyAsync(evh.data(), h->ev, k * sizeof(cplx), cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaStreamSynchronize(s));
        std::vector<std::complex<double>> th(k);
        for (int i = 0; i < k; ++i) th[i] = {evh[i].x, evh[i].y};
        const int idx = pick_nearest_one(th);
        inf->ritz_value = th[idx].real();
        // Arnoldi residual estimate of the Ritz pair: |h_{k,k-1}| |y_{k-1}|
        cplx tail[2];
        LB_CHECK_CUDA(cudaMemcpyAsync(&tail[0], h->hm + (size_t)(k - 1) * h->ldh + k, sizeof(cplx),
                                      cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaMemcpyAsync(&tail[1], h->evec + (size_t)idx * k + k - 1, sizeof(cplx),
                                      cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaStreamSynchronize(s));
        const double ritz_res = std::hypot(tail[0].x, tail[0].y) * std::hypot(tail[1].x, tail[1].y);
        // xi = V y, phase-fixed by its trace
        if (vec_gemv(xi, h->V, nn, k, h->evec + (size_t)idx * k, nn, 1.0, 0, s)) return LB_CUDA_ERROR;
        if (mat_trace(xi, n, h->scal + 2, s)) return LB_CUDA_ERROR;
        if (mat_div_by_dev(xi, xi, nn, h->scal + 2, s)) return LB_CUDA_ERROR;
        bool reconstruct = true;
        if (prec == LB_PREC_MIXED) {
            // low-precision phase: iterate until the Ritz residual reaches the split-GEMM accuracy
            // floor or stops halving; the state is then reconstructed once and refined in FP64
            const bool stop = ritz_res < 1e-7 * std::abs(th[idx]) || (restart > 0 && ritz_res > 0.5 * prev_ritz) ||
                              restart + 1 == o.max_restarts;
            prev_ritz = std::min(prev_ritz, ritz_res);
            reconstruct = stop;
        }
        if (reconstruct) {
            // rho~ = -S~^{-1} xi, hermitised and trace-normalised
            if (lyap_schur(h, s, xi, rt, 0.0, prec)) return LB_CUDA_ERROR;
            if (hermitize_normalize(h, s, rt, rt, R)) return LB_CUDA_ERROR;
            if (change_basis(h, s, rt, rho, R, 0)) return LB_CUDA_ERROR;
            // the returned state is hermitised and trace-normalised in the original basis
            if (hermitize_normalize(h, s, rho, rho, R)) return LB_CUDA_ERROR;
            double rmax, rfro;
            if (residual_norms(h, s, rho, R, &rmax, &rfro)) return LB_CUDA_ERROR;
            if (rmax < best) {
                best = rmax;
                inf->residual_max = rmax;
                inf->residual_fro = rfro;
                LB_CHECK_CUDA(cudaMemcpyAsync(rho_out, rho, nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
                LB_CHECK_CUDA(cudaMemcpyAsync(h->best, rt, nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
                LB_CHECK_CUDA(cudaMemcpyAsync(h->Rres, R, nn * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
            }
            if (rmax < o.tol || prec == LB_PREC_MIXED) { ++restart; break; }
        }
        // restart from xi (unit norm)
        if (vec_norms(xi, nn, h->dpart, h->dscal, s)) return LB_CUDA_ERROR;
        double nr[2];
        LB_CHECK_CUDA(cudaMemcpyAsync(nr, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        LB_CHECK_CUDA(cudaStreamSynchronize(s));
        if (!(nr[1] > 0.0)) break;
        if (vec_scale_copy(h->V, xi, nn, cmake(1.0 / nr[1], 0.0), s)) return LB_CUDA_ERROR;
    }
    inf->restarts = restart;
    LB_CHECK_CUDA(cudaStreamSynchronize(s));
    return inf->residual_max < o.tol ? LB_OK : LB_NOT_CONVERGED;
}
