// Tensor-core complex GEMM on split FP16 planes (sm_103a: TMA + tcgen05.mma + TMEM).
//
// An FP64 complex matrix X is stored for the tensor cores as four FP16 planes
// [re_hi, re_lo, im_hi, im_lo] with X ~ 2^-e (hi + lo) (e a per-matrix power-of-two scale),
// so that each product term carries ~22 significant bits.  One complex product over K is
// accumulated in FP32 in TMEM as
//     Dr += Ar Br^T - Ai Bi^T,   Di += Ar Bi^T + Ai Br^T
// over the split pairs (hi,hi), (hi,lo), (lo,hi) -- the "4-real" complex product, three
// split terms each.  Operands are K-major (row r of a plane holds op(X)[r, 0..K)).
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace tc {

constexpr int BM = 128;   // tile rows (MMA M)
constexpr int BN = 128;   // tile cols (MMA N)
constexpr int BK = 64;    // K per stage: 64 fp16 = one 128-byte swizzle row
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 2;              // 16 KiB (BM == BN)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;          // A re, A im, B re, B im
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int MAX_SEGS = 2;

// sign conventions of one segment
enum { SIGN_NORMAL = 0, SIGN_CONJ_B = 1, SIGN_CONJ_A = 2 };

struct Seg {
    int a_map, b_map;        // tensor-map slots
    int a_row, b_row;        // row-coordinate offsets added to the tile origin (m0 / n0)
    int a_j, b_j;            // batch (dim 2) coordinate of the first K-batch
    int a_jstep, b_jstep;    // batch step per K-batch
    int nbatch;              // number of K-batches
    int k0, klen;            // K range (dim 0) within each batch
    int sign;                // SIGN_*
};

struct Maps {
    CUtensorMap m[4];
};

struct Params {
    int M, N;                // output extent (rows, cols) -- masks the epilogue
    int nseg;
    Seg seg[MAX_SEGS];
    int npairs;              // 1: (hi,hi) only; 3: (hi,hi),(hi,lo),(lo,hi)
    // epilogue: out[r * ldo + c] = alpha * scale[0] * (Dr + i Di) (+ beta * out)
    cplx* out;
    long long ldo;
    double alpha;
    const double* scale;     // device scalar (product of the operands' inverse scales), nullable
    int accumulate;          // 1: out += result
    int* err;                // device error word (set on a wait timeout)
    int fmt;                 // operand format: 0 FP16, 1 BF16
    // wavefront mode (triangular Sylvester updates): wave >= 0 maps CTA b to the block
    // (I, J) = (nb-1-t, nb-1-(wave-t)), t = b + max(0, wave-(nb-1)); segment 0 then runs
    // over K in [(I+1) BM, nb BM) and segment 1 over [(J+1) BN, nb BN)
    int wave;
    int nb;
    // ksplit > 1: the K range of each output tile (all segments and batches, in BK blocks) is split
    // into ksplit chunks run by separate CTAs (chunk = blockIdx.y in wavefront mode, blockIdx.z
    // otherwise); partial products are added to out with FP64 atomics (out must hold the addend, e.g.
    // zeros); not with the planes epilogue
    int ksplit;
    // 1: the output is Hermitian (M = N); tiles strictly below the diagonal exit at once and are
    // mirrored by the caller
    int tri;
    // non-null: instead of complex128 `out`, the epilogue writes the result (times scale[0] and alpha) as
    // the four FP16 planes [re_hi, re_lo, im_hi, im_lo] of the next product's operand: plane q at
    // planes + q * plane_stride, row r at r * plane_ld; every row < M and column < N is written (zeros
    // included), so the padding of the planes is kept zero
    __half* planes;
    long long plane_stride;
    int plane_ld;
    // limit of every mbarrier wait in ns (0: 2 s); a wait that runs out sets *err and its role gives up
    unsigned long long wait_ns;
    // test of the bounded waits: s > 0 makes the TMA producer issue no loads for its iteration s - 1,
    // so the MMA issuer's wait for that stage runs out (0: normal operation)
    int test_stall;
};

}  // namespace tc

// host-side helpers (tc_gemm.cu)
// planes: 4 * nbatch * rows * ld halves, plane-major; builds a 4D map (K, rows, nbatch, 4)
int tc_make_map(CUtensorMap* map, const void* planes, int K, int rows, int nbatch, int ld, int bf16 = 0);
int tc_gemm_launch(const tc::Maps& maps, const tc::Params& p, int grid_m, int grid_n, cudaStream_t s);
// X (complex128, rows x cols, ld_src) -> 4 FP16 planes (rows x ld_dst, plane stride pstride),
// element op: transpose (op = 1) / conjugate (conj = 1); value scaled by scale_dev[0].
int tc_split_planes(const cplx* X, long long ld_src, int rows, int cols, int transpose, int conj,
                    const double* scale_dev, __half* planes, int ld_dst, long long pstride, int batch,
                    long long src_bstride, long long dst_bstride, cudaStream_t s);
// the same packing into BF16 hi/lo planes, no scale
int tc_split_planes_bf16(const cplx* X, long long ld_src, int rows, int cols, int transpose, void* planes,
                         int ld_dst, long long pstride, cudaStream_t s);
// out[0] = max over the len complex entries of max(|re|, |im|); part: >= 592 doubles of scratch
int tc_maxabs(const cplx* X, long long len, double* part, double* out, cudaStream_t s);
// scale_dev[0] = 2^e with 2^e * maxabs <= 2^14 ; inv_dev[0] = 2^-e  (maxabs from tc_maxabs)
// the largest row 1-norm sum_k (|Re A_rk| + |Im A_rk|) over the rows of A (rows x cols, ld), to out[0]
int tc_max_row_l1(const cplx* A, long long rows, int cols, long long ld, double* part, double* out, cudaStream_t s);
// scale_dev[0] = 2^e with 2^e * a[0] * b[0] * sqrt(2) <= 2^14 (a bound on the next product's entries),
// inv_dev[0] = 2^-e, fac_dev[0] = scale * c[0] (c: the product of the operands' inverse scales)
int tc_bound_scale(const double* a, const double* b, const double* c, double* scale_dev, double* inv_dev,
                   double* fac_dev, cudaStream_t s);
int tc_pick_scale(const double* maxabs_dev, double* scale_dev, double* inv_dev, cudaStream_t s);
