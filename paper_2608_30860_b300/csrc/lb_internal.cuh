// Internal state of a lindblad_handle and the host-side sequencing helpers shared between
// lindblad.cu (set-up, Phi, Alg. 4), solvers.cu (GMRES, refinement, Alg. 5) and
// mixed.cu (tensor-core path).
#pragma once
#include <functional>
#include <vector>

#include "../../include/lindblad.h"
#include "common.cuh"

#define LB_CHECK_CUDA(expr)                                                                 \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            fprintf(stderr, "lindblad: CUDA error %s at %s:%d\n", cudaGetErrorString(_e),   \
                    __FILE__, __LINE__);                                                    \
            return LB_CUDA_ERROR;                                                           \
        }                                                                                   \
    } while (0)

constexpr int KMAX = 64;      // largest Krylov cycle (outer Arnoldi or inner GMRES)
constexpr int NSCRATCH = 8;   // n x n scratch matrices

struct MixedState;            // tensor-core jump-term buffers (mixed.cu)
struct SylvMixed;             // tensor-core triangular Sylvester buffers (sylv_mixed.cu)

struct lb_handle_s {
    int n = 0, d = 0;
    lb_opts opts{};
    size_t ws_bytes = 0;
    // FP64 problem data and factors (device)
    cplx *H = nullptr, *L = nullptr, *G = nullptr, *Q = nullptr, *T = nullptr, *Lt = nullptr;
    cplx* P = nullptr;                 // d n^2 scratch (jump-term intermediate)
    cplx* X[NSCRATCH] = {};            // n x n scratch
    cplx* best = nullptr;              // n x n
    // recycled GMRES (recycle.cu): pair (U^, C) with B U^ = C diag(dU), U^ unit columns, C orthonormal
    int rk = 0;                        // capacity (vectors)
    cplx *Urc = nullptr, *Crc = nullptr, *Unw = nullptr, *Cnw = nullptr;
    double* dU = nullptr;              // 2 x 16: current and next scale factors
    cplx* gsm = nullptr;               // small dense matrices of the GCRO-DR cycle
    int rc_have = 0;                   // size of the pair in use (0: none)
    double rc_mu = 0.0, rc_eta = 0.0;  // operator the pair belongs to
    int rc_prec = -1;
    cplx* Rres = nullptr;              // L(rho) of the accepted steady-state iterate (original basis)
    cplx* bk0 = nullptr;               // backups of the accepted iterate during refinement
    cplx* bk1 = nullptr;
    cplx* W = nullptr;                 // R_mu^S(I) for the Sherman-Morrison preconditioner
    cplx* Wa = nullptr;                // its adjoint counterpart R_mu^{S*}(I)
    cplx* Ua = nullptr;                // J T^dag J (J = index reversal): upper triangular, adjoint solves
    cplx* Re = nullptr;                // R = Q^dag U (eigenbasis route), upper triangular
    cplx* Rinv = nullptr;              // R^{-1}
    cplx* E1 = nullptr;                // eigenbasis-route scratch (n x n each)
    cplx* E2 = nullptr;
    bool eig_active = false;           // FP64 Lyapunov solves use the eigenbasis route
    int arn_depth = 0;                 // nesting level of arnoldi_cycle (breakdown flag dinfo[12 + level])
    unsigned long long tc_wait_ns = 0; // limit of the tensor-core kernels' mbarrier waits (0: 2 s)
    int tc_stall = 0;                  // bounded-wait test: stall iteration + 1 of the next jump product (1)
    bool gauged = false;               // H, L hold the gauge-shifted H~, L~_j (lb_opts.gauge_c)
    double cond_eig = 0.0;
    bool ua_ready = false;
    cplx* V = nullptr;                 // inner Krylov basis (vcap vectors)
    cplx* Z = nullptr;                 // outer Krylov basis (vcap vectors)
    int vcap = 0;
    cplx* hm = nullptr;                // (KMAX+1) x (KMAX+1) column-major, ld = ldh (inner)
    cplx* hm2 = nullptr;               // same, outer
    int ldh = 0;
    cplx* ev = nullptr;                // KMAX
    cplx* evec = nullptr;              // KMAX x KMAX
    cplx* small = nullptr;             // 4 (KMAX+2)
    cplx* part = nullptr;              // DOT_BLOCKS (KMAX+2)
    double* dpart = nullptr;           // 2 DOT_BLOCKS
    double* dscal = nullptr;           // 16
    cplx* scal = nullptr;              // 16
    int* dinfo = nullptr;              // 16
    char* solver_ws = nullptr;
    size_t solver_ws_bytes = 0;
    char* mixed_base = nullptr;
    MixedState* mixed = nullptr;
    SylvMixed* sylv = nullptr;
    bool mixed_ready = false;         // tensor-core jump term available
    bool mixed_sylv_ready = false;    // tensor-core triangular Sylvester available
    // host-side diagnostics
    double gnorm = 0.0, schur_err = 0.0, min_re_T = 0.0, setup_ms = 0.0;
    int case1 = 0;
    // kernel timing (lb_set_profiling): event pairs and algorithmic flops per kernel id
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev[2];
    std::vector<double> prof_flops[2];
    ~lb_handle_s();
};

typedef std::function<int(const cplx*, cplx*)> OpFn;

// lindblad.cu
// kernel timing hooks: record an event pair around a launch when profiling is on
void prof_begin(lb_handle_s* h, cudaStream_t s, int kid);
void prof_end(lb_handle_s* h, cudaStream_t s, int kid, double flops);
int gemm(lb_handle_s* h, cudaStream_t s, cplx* C, const cplx* A, int opA, const cplx* B, int opB, int M, int N,
         int K, cplx alpha, cplx beta);
int jump_f64(lb_handle_s* h, cudaStream_t s, const cplx* Ls, const cplx* Z, cplx* Y, cplx alpha, cplx beta,
             int herm = 0);
int lindbladian_f64(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* R);
int lindbladian_f64_herm(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* R);
int change_basis(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* Out, cplx* tmp, int to_schur);
int lyap_schur(lb_handle_s* h, cudaStream_t s, const cplx* Y, cplx* X, double shift, int precision);
int lyap_eig(lb_handle_s* h, cudaStream_t s, const cplx* Y, cplx* X, double shift);
int phi_schur(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* Y, int form, int precision, int herm = 0);
int arnoldi_cycle(lb_handle_s* h, cudaStream_t s, cplx* basis, cplx* hess, int j0, int m, const OpFn& op,
                  int* k_out);
int hermitize_normalize(lb_handle_s* h, cudaStream_t s, const cplx* in, cplx* out, cplx* tmp);
int residual_norms(lb_handle_s* h, cudaStream_t s, const cplx* rho, cplx* R, double* rmax, double* rfro);
lb_status check_device_error(lb_handle_s* h, cudaStream_t s);
lb_status device_error_guard(lb_handle_s* h, cudaStream_t s, lb_status st);
lb_status steady_state_arnoldi(lb_handle_s* h, cudaStream_t s, const lb_opts& o, cplx* rho_out, lb_info* inf);

// solvers.cu
lb_status precond_prepare(lb_handle_s* h, cudaStream_t s, double mu, double eta, int precision, int adj);
int precond_apply(lb_handle_s* h, cudaStream_t s, const cplx* X, cplx* out, double mu, double eta, int precision,
                  int adj);
int pure_state_case1(lb_handle_s* h, cudaStream_t s, cplx* rho_out);
lb_status refine_steady_state(lb_handle_s* h, cudaStream_t s, const lb_opts& o, cplx* rho, lb_info* inf);

lb_status adj_precond_prepare(lb_handle_s* h, cudaStream_t s, double eta);
int adj_gmres_solve(lb_handle_s* h, cudaStream_t s, const cplx* b, cplx* x, double eta, int m, int max_cycles,
                    double atol, int* steps, double* final_res);

// recycle.cu
size_t recycle_bytes(int n, int rk);
void recycle_layout(lb_handle_s* h, char*& base, int rk);
void recycle_forget(lb_handle_s* h);
int gcrodr_solve(lb_handle_s* h, cudaStream_t s, const cplx* b, cplx* delta, double mu, double eta, int m, int kreq,
                 int max_cycles, double atol, int precision, int* steps, double* final_res, int* cycles_out);

// adjoint.cu
int adj_lyap_schur(lb_handle_s* h, cudaStream_t s, const cplx* Y, cplx* X, double shift);
int adj_jump_f64(lb_handle_s* h, cudaStream_t s, const cplx* Z, cplx* Y, cplx alpha, cplx beta);

// mixed.cu
size_t mixed_bytes(int n, int d);
size_t mixed_P_rows(int n, int d);
int mixed_prepare(lb_handle_s* h, cudaStream_t s);
int jump_mixed(lb_handle_s* h, cudaStream_t s, const cplx* Z, cplx* Y, double alpha, int herm = 0);
void mixed_release(lb_handle_s* h);

// sylv_mixed.cu
size_t sylv_mixed_bytes(int n);
int sylv_mixed_prepare(lb_handle_s* h, char* base, cudaStream_t s);
int trisylv_mixed(lb_handle_s* h, cudaStream_t s, cplx* X, double shift);
void sylv_mixed_release(lb_handle_s* h);
