// Mixed-precision (tensor-core) jump term in Schur coordinates:
//   K~(Z) = sum_j L~_j Z L~_j^dag
// as two split-FP16 complex GEMMs on tcgen05 (tc_gemm.cu), FP32 accumulation:
//   (1) P = [L~_1; ...; L~_d] Z          one stacked product, M = d * n_pad, whose epilogue writes P
//                                        directly as the FP16 hi/lo planes of product (2)'s operand
//   (2) Y = alpha sum_j P_j L~_j^dag     one product whose K loop runs over (j, k); for Hermitian Z the
//                                        tiles below the diagonal are skipped and mirrored
// The L~_j planes are packed once at set-up; Z is packed per call with a power-of-two scale
// (max |entry| -> 2^14); P's scale comes from the bound max_r ||L~_r,:||_1 sqrt(2) max|Z| (P is never
// stored in FP64), and the epilogues undo the scales.
#include <algorithm>

#include "lb_internal.cuh"
#include "tc_gemm.cuh"
#include "vecops.cuh"

struct MixedState {
    int np = 0;                   // n rounded up to the 128-row tile
    __half* Lp = nullptr;         // 4 x d x np x np
    __half* Zp = nullptr;         // 4 x np x np
    __half* Pp = nullptr;         // 4 x d x np x np
    double* sc = nullptr;         // scales: see below
    tc::Maps maps{};              // 0: L stack (rows d*np), 1: Z, 2: P (batch d), 3: L (batch d)
};

// sc[0] scale_L, sc[1] inv_L, sc[2] scale_Z, sc[3] inv_Z, sc[4] scale_P, sc[5] inv_P,
// sc[6] inv_L*inv_Z, sc[7] inv_P*inv_L, sc[8] max|Z| (re/im), sc[9] scratch,
// sc[10] the factor product (1)'s epilogue applies (scale_P inv_L inv_Z),
// sc[11] max_{j,r} sum_k (|Re L~_j[r,k]| + |Im L~_j[r,k]|) (set-up)
namespace {

constexpr int KSPLIT2 = 4;   // CTAs per output tile of product (2)

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

__global__ void k_mul2(double* out, const double* a, const double* b) {
    if (threadIdx.x == 0) out[0] = a[0] * b[0];
}

}  // namespace

size_t mixed_bytes(int n, int d) {
    const size_t np = (size_t)round_up(n, tc::BM);
    const size_t planes1 = 4 * np * np * sizeof(__half);
    return (size_t)d * planes1 + planes1 + (size_t)d * planes1 + 64 * sizeof(double) + 4 * 256 + sylv_mixed_bytes(n);
}

size_t mixed_P_rows(int n, int d) { return (size_t)d * round_up(n, tc::BM); }

int mixed_prepare(lb_handle_s* h, cudaStream_t s) {
    const int n = h->n, d = h->d;
    MixedState* m = new MixedState();
    h->mixed = m;
    m->np = round_up(n, tc::BM);
    const size_t np = m->np;
    char* base = h->mixed_base;
    auto carve = [&](size_t bytes) {
        char* p = base;
        base += (bytes + 255) & ~size_t(255);
        return p;
    };
    m->Lp = reinterpret_cast<__half*>(carve(4 * (size_t)d * np * np * sizeof(__half)));
    m->Zp = reinterpret_cast<__half*>(carve(4 * np * np * sizeof(__half)));
    m->Pp = reinterpret_cast<__half*>(carve(4 * (size_t)d * np * np * sizeof(__half)));
    m->sc = reinterpret_cast<double*>(carve(64 * sizeof(double)));
    // L~ planes with one scale for the whole stack
    if (tc_maxabs(h->Lt, (long long)d * n * n, h->dpart, m->sc + 8, s)) return -1;
    if (tc_pick_scale(m->sc + 8, m->sc + 0, m->sc + 1, s)) return -1;
    if (tc_split_planes(h->Lt, n, n, n, 0, 0, m->sc + 0, m->Lp, (int)np, (long long)d * np * np, d,
                        (long long)n * n, (long long)np * np, s))
        return -1;
    // the a-priori bound |P_rc| <= max_r ||L~_j[r,:]||_1 sqrt(2) max|Z| that scales P's planes
    if (tc_max_row_l1(h->Lt, (long long)d * n, n, n, h->dpart, m->sc + 11, s)) return -1;
    if (tc_make_map(&m->maps.m[0], m->Lp, (int)np, (int)(d * np), 1, (int)np)) return -1;
    if (tc_make_map(&m->maps.m[1], m->Zp, (int)np, (int)np, 1, (int)np)) return -1;
    if (tc_make_map(&m->maps.m[2], m->Pp, (int)np, (int)np, d, (int)np)) return -1;
    if (tc_make_map(&m->maps.m[3], m->Lp, (int)np, (int)np, d, (int)np)) return -1;
    h->mixed_ready = true;
    return sylv_mixed_prepare(h, base, s);
}

// Y = alpha * sum_j L~_j Z L~_j^dag  (Z, Y: n x n complex128, Schur coordinates).  herm = 1 (Z Hermitian):
// product (2) is Hermitian, its tiles below the diagonal are skipped and mirrored.
int jump_mixed(lb_handle_s* h, cudaStream_t s, const cplx* Z, cplx* Y, double alpha, int herm) {
    MixedState* m = h->mixed;
    if (!m) return -1;
    const int n = h->n, d = h->d, np = m->np;
    int* err = h->dinfo + 8;
    // pack Z^T (the B operand of product (1) is K-major: row c holds column c of Z)
    if (tc_maxabs(Z, (long long)n * n, h->dpart, m->sc + 8, s)) return -1;
    if (tc_pick_scale(m->sc + 8, m->sc + 2, m->sc + 3, s)) return -1;
    if (tc_split_planes(Z, n, n, n, 1, 0, m->sc + 2, m->Zp, np, (long long)np * np, 1, 0, (long long)np * np, s))
        return -1;
    k_mul2<<<1, 32, 0, s>>>(m->sc + 6, m->sc + 1, m->sc + 3); lb_note_launch();
    // scale of P from the bound, and the epilogue factor scale_P inv_L inv_Z
    if (tc_bound_scale(m->sc + 11, m->sc + 8, m->sc + 6, m->sc + 4, m->sc + 5, m->sc + 10, s)) return -1;
    // (1) P = L~_stack Z, written by the epilogue straight into the FP16 hi/lo planes that product (2)
    // reads (d np rows of P_j, K-major as stored; padding rows and columns written as zeros)
    tc::Params p1{};
    p1.M = d * np;
    p1.N = np;
    p1.nseg = 1;
    p1.seg[0] = tc::Seg{0, 1, 0, 0, 0, 0, 0, 0, 1, 0, np, tc::SIGN_NORMAL};
    p1.npairs = 3;
    p1.out = nullptr;
    p1.ldo = 0;
    p1.alpha = 1.0;
    p1.scale = m->sc + 10;
    p1.accumulate = 0;
    p1.err = err;
    p1.fmt = 0;
    p1.wave = -1;
    p1.planes = m->Pp;
    p1.plane_stride = (long long)d * np * np;
    p1.plane_ld = np;
    p1.wait_ns = h->tc_wait_ns;
    p1.test_stall = h->tc_stall;
    h->tc_stall = 0;   // one launch only
    prof_begin(h, s, 0);
    if (tc_gemm_launch(m->maps, p1, d * np / tc::BM, np / tc::BN, s)) return -1;
    prof_end(h, s, 0, 8.0 * d * (double)n * n * n);
    k_mul2<<<1, 32, 0, s>>>(m->sc + 7, m->sc + 5, m->sc + 1); lb_note_launch();
    // (2) Y = alpha sum_j P_j conj(L~_j)^T  : B rows are conj(L~_j) rows
    tc::Params p2{};
    p2.M = n;
    p2.N = n;
    p2.nseg = 1;
    p2.seg[0] = tc::Seg{2, 3, 0, 0, 0, 0, 1, 1, d, 0, np, tc::SIGN_CONJ_B};
    p2.npairs = 3;
    p2.out = Y;
    p2.ldo = n;
    p2.alpha = alpha;
    p2.scale = m->sc + 7;
    p2.accumulate = 0;
    p2.err = err;
    p2.fmt = 0;
    p2.wave = -1;
    p2.tri = herm;
    // the K loop of (2) runs over d n products: split it over KSPLIT2 CTAs per tile (whole jumps per
    // chunk when KSPLIT2 divides d), partial sums added in FP64 -- each FP32 accumulation chain is
    // KSPLIT2 times shorter, and small n fills the SMs
    p2.ksplit = std::min(d, KSPLIT2);
    p2.wait_ns = h->tc_wait_ns;
    prof_begin(h, s, 0);
    if (p2.ksplit > 1 && cudaMemsetAsync(Y, 0, (size_t)n * n * sizeof(cplx), s) != cudaSuccess) return -1;
    int r = tc_gemm_launch(m->maps, p2, (n + tc::BM - 1) / tc::BM, (n + tc::BN - 1) / tc::BN, s);
    if (!r && herm) r = mat_mirror_lower(Y, n, n, s, herm == 2);
    // algorithmic work: the full product, or its Hermitian half (n (n + 1) / 2 entries)
    prof_end(h, s, 0, (herm ? 4.0 * (n + 1) : 8.0 * n) * d * (double)n * n);
    return r;
}

void mixed_release(lb_handle_s* h) {
    delete h->mixed;
    h->mixed = nullptr;
    sylv_mixed_release(h);
}

lb_handle_s::~lb_handle_s() { mixed_release(this); }
