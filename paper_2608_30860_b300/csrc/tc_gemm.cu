// Tensor-core complex GEMM kernel (tcgen05 + TMA + TMEM, sm_103a) and its operand packing.
//
// CTA = 8 warps, one 128 x 128 output tile (real and imaginary accumulators, 256 TMEM columns):
//   warp 0 (lane 0) : TMA producer -- per stage the four 128 x 64 FP16 tiles A_re, A_im, B_re,
//                     B_im (128-byte swizzle), one mbarrier with the byte count;
//   warp 1 (lane 0) : MMA issuer -- 16 tcgen05.mma (M128 N128 K16) per stage, then
//                     tcgen05.commit to the stage's "empty" barrier; warp 1 also owns TMEM;
//   warps 4..7      : epilogue -- tcgen05.ld of the FP32 accumulators (each warp its 32-lane
//                     quarter), scaling, FP64 complex store.
// Three-stage ring.  Every mbarrier wait is bounded (2 s of %globaltimer unless Params::wait_ns says
// otherwise); a timeout sets the error word and the roles fall through to the TMEM release.
#include <cuda.h>
#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace tc {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok;
}
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (gtimer() - t0 > limit_ns) {
            atomicExch(err, code);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor, kind::f16: D = F32 (bits 4-5), A = B = F16 (bits 7-9, 10-12),
// both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24; bit 13 negates A.
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t NEG_A = 1u << 13;

__device__ __forceinline__ int seg_iters(const Seg& sg, int npairs) {
    return sg.klen > 0 ? sg.nbatch * ((sg.klen + BK - 1) / BK) * npairs : 0;
}

// segment g of this CTA (wavefront mode adjusts the K ranges to the block (I, J))
__device__ __forceinline__ Seg cta_seg(const Params& p, int g, int I, int J) {
    Seg sg = p.seg[g];
    if (p.wave >= 0) {
        const int lo = (g == 0 ? I + 1 : J + 1) * BM;
        sg.k0 = lo;
        sg.klen = p.nb * BM - lo;
    }
    return sg;
}

__global__ void __launch_bounds__(256, 1) k_tc_gemm(const __grid_constant__ Maps maps,
                                                    const __grid_constant__ Params p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char* smem = smem_raw + pad;
    const uint32_t sbase = raw + pad;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    const uint32_t full0 = smem_u32(bars);
    const uint32_t empty0 = full0 + 8 * STAGES;
    const uint32_t accf = full0 + 16 * STAGES;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, I = 0, J = 0;
    if (p.wave < 0) {
        // grouped raster: consecutive CTAs walk a band of GROUP_M row tiles across all column tiles,
        // so the ~148 resident CTAs share ~12 row tiles and ~12 column tiles of the operands in L2
        // (with the plain x-fastest order every column tile re-read all of A from DRAM)
        constexpr int GROUP_M = 12;
        const int lin = blockIdx.y * gridDim.x + blockIdx.x;
        const int per_group = GROUP_M * gridDim.y;
        const int g0 = (lin / per_group) * GROUP_M;
        const int gm = min(GROUP_M, (int)gridDim.x - g0);
        const int local = lin % per_group;
        m0 = (g0 + local % gm) * BM;
        n0 = (local / gm) * BN;
    }
    if (p.wave >= 0) {
        const int t = blockIdx.x + max(0, p.wave - (p.nb - 1));
        I = p.nb - 1 - t;
        J = p.nb - 1 - (p.wave - t);
        m0 = I * BM;
        n0 = J * BN;
    }
    // Hermitian output: the CTAs of tiles strictly below the diagonal leave before any set-up
    if (p.tri && m0 > n0) return;
    // K units (batch x BK block) of this CTA: all of them, or chunk c of ksplit (c = blockIdx.y in
    // wavefront mode, blockIdx.z otherwise); split partial products are added to out with FP64 atomics
    const bool split = p.ksplit > 1 && !p.planes;
    int u_lo = 0, u_hi = 0x7fffffff;
    if (split) {
        const int chunk = p.wave >= 0 ? (int)blockIdx.y : (int)blockIdx.z;
        int units = 0;
        for (int g = 0; g < p.nseg; ++g) units += seg_iters(cta_seg(p, g, I, J), 1);
        u_lo = (int)((long long)units * chunk / p.ksplit);
        u_hi = (int)((long long)units * (chunk + 1) / p.ksplit);
    }
    int total_iters = 0;
    {
        int u = 0;
        for (int g = 0; g < p.nseg; ++g) {
            const int nu = seg_iters(cta_seg(p, g, I, J), 1);
            const int lo = max(u, u_lo), hi = min(u + nu, u_hi);
            if (hi > lo) total_iters += (hi - lo) * p.npairs;
            u += nu;
        }
    }
    const uint32_t idesc_base = IDESC | ((uint32_t)p.fmt << 7) | ((uint32_t)p.fmt << 10);
    const uint64_t limit = p.wait_ns ? p.wait_ns : 2000000000ull;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accf, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int i = 0; i < 4; ++i)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.m[i])) : "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), 2 * BN);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- TMA producer
        int it = 0, u = 0;
        bool ok = true;
        for (int g = 0; g < p.nseg && ok; ++g) {
            const Seg sg = cta_seg(p, g, I, J);
            if (sg.klen <= 0) continue;
            const int nkb = (sg.klen + BK - 1) / BK;
            const CUtensorMap* am = &maps.m[sg.a_map];
            const CUtensorMap* bm = &maps.m[sg.b_map];
            for (int jb = 0; jb < sg.nbatch && ok; ++jb) {
                const int aj = sg.a_j + jb * sg.a_jstep, bj = sg.b_j + jb * sg.b_jstep;
                for (int kb = 0; kb < nkb && ok; ++kb, ++u) {
                    if (u < u_lo || u >= u_hi) continue;
                    const int kc = sg.k0 + kb * BK;
                    for (int pr = 0; pr < p.npairs; ++pr, ++it) {
                        if (it + 1 == p.test_stall) continue;   // no loads: the stage never fills
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1;
                        if (!mbar_wait(empty0 + 8 * s, ph ^ 1, p.err, 1, limit)) { ok = false; break; }
                        const int sa = (pr == 2) ? 1 : 0, sb = (pr == 1) ? 1 : 0;
                        const uint32_t st = sbase + s * STAGE_BYTES;
                        const uint32_t fb = full0 + 8 * s;
                        mbar_expect_tx(fb, STAGE_BYTES);
                        tma_load_4d(st, am, fb, kc, m0 + sg.a_row, aj, sa);
                        tma_load_4d(st + TILE_BYTES, am, fb, kc, m0 + sg.a_row, aj, 2 + sa);
                        tma_load_4d(st + 2 * TILE_BYTES, bm, fb, kc, n0 + sg.b_row, bj, sb);
                        tma_load_4d(st + 3 * TILE_BYTES, bm, fb, kc, n0 + sg.b_row, bj, 2 + sb);
                    }
                }
            }
        }
        // drain: the loads of the last (up to STAGES) issued stages must have landed
        for (int q = (it > STAGES ? it - STAGES : 0); q < it; ++q)
            mbar_wait(full0 + 8 * (q % STAGES), (q / STAGES) & 1, p.err, 4, limit);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        int it = 0, u = 0;
        bool ok = true;
        for (int g = 0; g < p.nseg && ok; ++g) {
            const Seg sg = cta_seg(p, g, I, J);
            const uint32_t id_rr = idesc_base;
            const uint32_t id_ii = (sg.sign == SIGN_NORMAL) ? (idesc_base | NEG_A) : idesc_base;
            const uint32_t id_ri = (sg.sign == SIGN_CONJ_B) ? (idesc_base | NEG_A) : idesc_base;
            const uint32_t id_ir = (sg.sign == SIGN_CONJ_A) ? (idesc_base | NEG_A) : idesc_base;
            const int nu = seg_iters(sg, 1);
            const int lo = max(u, u_lo) - u, hi = min(u + nu, u_hi) - u;
            u += nu;
            const int n_it = hi > lo ? (hi - lo) * p.npairs : 0;
            for (int q = 0; q < n_it; ++q, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!mbar_wait(full0 + 8 * s, ph, p.err, 2, limit)) { ok = false; break; }
                fence_after();
                const uint32_t st = sbase + s * STAGE_BYTES;
                const uint64_t dAr = desc_sw128(st), dAi = desc_sw128(st + TILE_BYTES);
                const uint64_t dBr = desc_sw128(st + 2 * TILE_BYTES), dBi = desc_sw128(st + 3 * TILE_BYTES);
#pragma unroll
                for (int t = 0; t < BK / 16; ++t) {
                    const uint64_t off = (uint64_t)((t * 32) >> 4);   // 16 fp16 = 32 bytes along K
                    const uint32_t acc = (it == 0 && t == 0) ? 0u : 1u;
                    umma(tmem, dAr + off, dBr + off, id_rr, acc);
                    umma(tmem, dAi + off, dBi + off, id_ii, 1u);
                    umma(tmem + BN, dAr + off, dBi + off, id_ri, acc);
                    umma(tmem + BN, dAi + off, dBr + off, id_ir, 1u);
                }
                umma_commit(empty0 + 8 * s);
            }
        }
        if (total_iters > 0) umma_commit(accf);
    } else if (warp >= 4 && total_iters > 0) {
        // ---------------------------------------------------------------- epilogue
        const int wq = warp - 4;
        const bool ok = mbar_wait(accf, 0, p.err, 3, limit);
        fence_after();
        const int r = m0 + wq * 32 + lane;
        const double sc = p.alpha * (p.scale ? p.scale[0] : 1.0);
        const uint32_t lane_addr = tmem + ((uint32_t)(wq * 32) << 16);
        for (int c = 0; c < BN; c += 32) {
            uint32_t vr[32], vi[32];
            tmem_ld32(lane_addr + c, vr);
            tmem_ld32(lane_addr + BN + c, vi);
            tmem_ld_wait();
            if (ok && r < p.M && p.planes) {
                // FP16 hi/lo planes of the scaled result (the split in FP32: the scale is a power of two)
                const float fs = (float)sc;
                __half* base = p.planes + (long long)r * p.plane_ld + n0 + c;
#pragma unroll
                for (int t0 = 0; t0 < 32; t0 += 8) {
                    if (n0 + c + t0 >= p.N) break;
                    __align__(16) __half hr[8], lr[8], hi_[8], li[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float re = __uint_as_float(vr[t0 + t]) * fs, im = __uint_as_float(vi[t0 + t]) * fs;
                        hr[t] = __float2half_rn(re);
                        lr[t] = __float2half_rn(re - __half2float(hr[t]));
                        hi_[t] = __float2half_rn(im);
                        li[t] = __float2half_rn(im - __half2float(hi_[t]));
                    }
                    *reinterpret_cast<uint4*>(base + t0) = *reinterpret_cast<const uint4*>(hr);
                    *reinterpret_cast<uint4*>(base + p.plane_stride + t0) = *reinterpret_cast<const uint4*>(lr);
                    *reinterpret_cast<uint4*>(base + 2 * p.plane_stride + t0) = *reinterpret_cast<const uint4*>(hi_);
                    *reinterpret_cast<uint4*>(base + 3 * p.plane_stride + t0) = *reinterpret_cast<const uint4*>(li);
                }
            } else if (ok && r < p.M) {
                cplx* orow = p.out + (long long)r * p.ldo;
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int col = n0 + c + t;
                    if (col < p.N) {
                        cplx v = cmake(sc * (double)__uint_as_float(vr[t]), sc * (double)__uint_as_float(vi[t]));
                        if (split) {
                            atomicAdd(&orow[col].x, v.x);
                            atomicAdd(&orow[col].y, v.y);
                        } else {
                            if (p.accumulate) v = cadd(v, orow[col]);
                            orow[col] = v;
                        }
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// ---------------------------------------------------------------- operand packing
// dst planes (plane-major): [re_hi, re_lo, im_hi, im_lo], each batch x rows_pad x ld_dst; the
// value op(X_b)[r][k] * scale is split as hi = fp16(v), lo = fp16(v - hi); padding is zero.
__global__ void k_split_planes(const cplx* __restrict__ X, long long ld_src, int rows, int cols, int transpose,
                               int conj, const double* __restrict__ scale_dev, __half* __restrict__ planes,
                               int ld_dst, int rows_pad, long long pstride, long long src_bstride,
                               long long dst_bstride) {
    __shared__ cplx tile[32][33];
    const int b = blockIdx.z;
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const float scf = scale_dev ? (float)scale_dev[0] : 1.0f;
    const cplx* Xb = X + (long long)b * src_bstride;
    // load the source tile so that global reads are coalesced
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        if (transpose) {
            // out[r][k] = X[k][r]: read rows k0+yy, columns r0+tx
            const int k = k0 + yy, r = r0 + threadIdx.x;
            tile[yy][threadIdx.x] = (k < cols && r < rows) ? Xb[(long long)k * ld_src + r] : cmake(0, 0);
        } else {
            const int r = r0 + yy, k = k0 + threadIdx.x;
            tile[yy][threadIdx.x] = (r < rows && k < cols) ? Xb[(long long)r * ld_src + k] : cmake(0, 0);
        }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int r = r0 + yy, k = k0 + threadIdx.x;
        if (r >= rows_pad || k >= ld_dst) continue;
        cplx v = transpose ? tile[threadIdx.x][yy] : tile[yy][threadIdx.x];
        // the split works in FP32: the scale is a power of two and hi + lo keep 22 of FP32's 24 bits,
        // so only the two conversions from FP64 use the (slow) FP64 pipe
        const float re = (float)v.x * scf, im = (conj ? -(float)v.y : (float)v.y) * scf;
        const __half rh = __float2half_rn(re), ih = __float2half_rn(im);
        const __half rl = __float2half_rn(re - __half2float(rh));
        const __half il = __float2half_rn(im - __half2float(ih));
        const long long o = (long long)b * dst_bstride + (long long)r * ld_dst + k;
        planes[o] = rh;
        planes[pstride + o] = rl;
        planes[2 * pstride + o] = ih;
        planes[3 * pstride + o] = il;
    }
}

// BF16 hi/lo planes, no scale (8-bit exponent): hi = bf16(v), lo = bf16(v - hi)
__global__ void k_split_planes_bf16(const cplx* __restrict__ X, long long ld_src, int rows, int cols, int transpose,
                                    __nv_bfloat16* __restrict__ planes, int ld_dst, int rows_pad, long long pstride) {
    __shared__ cplx tile[32][33];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        if (transpose) {
            const int k = k0 + yy, r = r0 + threadIdx.x;
            tile[yy][threadIdx.x] = (k < cols && r < rows) ? X[(long long)k * ld_src + r] : cmake(0, 0);
        } else {
            const int r = r0 + yy, k = k0 + threadIdx.x;
            tile[yy][threadIdx.x] = (r < rows && k < cols) ? X[(long long)r * ld_src + k] : cmake(0, 0);
        }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int r = r0 + yy, k = k0 + threadIdx.x;
        if (r >= rows_pad || k >= ld_dst) continue;
        const cplx v = transpose ? tile[threadIdx.x][yy] : tile[yy][threadIdx.x];
        const __nv_bfloat16 rh = __double2bfloat16(v.x), ih = __double2bfloat16(v.y);
        const __nv_bfloat16 rl = __double2bfloat16(v.x - (double)__bfloat162float(rh));
        const __nv_bfloat16 il = __double2bfloat16(v.y - (double)__bfloat162float(ih));
        const long long o = (long long)r * ld_dst + k;
        planes[o] = rh;
        planes[pstride + o] = rl;
        planes[2 * pstride + o] = ih;
        planes[3 * pstride + o] = il;
    }
}

// power-of-two scale with scale * maxabs <= 2^14
// max over the entries of max(|re|, |im|) from the bit patterns (for non-negative IEEE doubles the
// integer order is the numeric order), so no FP64 instruction is spent on it
__global__ void __launch_bounds__(256) k_maxabs_part(const unsigned long long* __restrict__ x, long long len,
                                                    unsigned long long* __restrict__ part) {
    __shared__ unsigned long long red[8];
    unsigned long long m = 0;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < len; e += (long long)gridDim.x * 256) {
        const unsigned long long b = __ldg(x + e) & 0x7fffffffffffffffull;
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < 8; ++q) m = red[q] > m ? red[q] : m;
        part[blockIdx.x] = m;
    }
}

__global__ void k_maxabs_final(const unsigned long long* __restrict__ part, int nblk, double* out) {
    unsigned long long m = 0;
    for (int b = threadIdx.x; b < nblk; b += 32) m = part[b] > m ? part[b] : m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if (threadIdx.x == 0) out[0] = __longlong_as_double((long long)m);
}

// per-block maxima of the row 1-norms sum_k (|Re| + |Im|), one warp per row
__global__ void k_row_l1_part(const cplx* __restrict__ A, long long rows, int cols, long long ld, double* part) {
    __shared__ double red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double m = 0.0;
    for (long long r = (long long)blockIdx.x * 8 + warp; r < rows; r += (long long)gridDim.x * 8) {
        double acc = 0.0;
        for (int k = lane; k < cols; k += 32) {
            const cplx v = A[r * ld + k];
            acc += fabs(v.x) + fabs(v.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        m = fmax(m, acc);
    }
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < 8; ++q) m = fmax(m, red[q]);
        part[blockIdx.x] = m;
    }
}

__global__ void k_max_part_final(const double* part, int nblk, double* out) {
    double m = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) m = fmax(m, part[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[0] = m;
}

// |(A B)_rc| <= max_r ||A_r,:||_1 max |B| and |B_kc| <= sqrt(2) max(|Re B_kc|, |Im B_kc|)
__global__ void k_bound_scale(const double* a, const double* b, const double* c, double* scale, double* inv,
                              double* fac) {
    if (threadIdx.x != 0) return;
    const double m = a[0] * b[0] * 1.4142135623730951;
    int e = 0;
    if (m > 0.0 && isfinite(m)) {
        frexp(m, &e);
        e = 14 - e;
    }
    scale[0] = ldexp(1.0, e);
    inv[0] = ldexp(1.0, -e);
    fac[0] = scale[0] * c[0];
}

__global__ void k_pick_scale(const double* maxabs, double* scale, double* inv) {
    if (threadIdx.x != 0) return;
    const double m = maxabs[0];
    int e = 0;
    if (m > 0.0 && isfinite(m)) {
        frexp(m, &e);            // m = f * 2^e, f in [0.5, 1)  => m < 2^e
        e = 14 - e;
    }
    scale[0] = ldexp(1.0, e);
    inv[0] = ldexp(1.0, -e);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

}  // namespace
}  // namespace tc

int tc_make_map(CUtensorMap* map, const void* planes, int K, int rows, int nbatch, int ld, int bf16) {
    tc::EncodeTiledFn fn = tc::encode_fn();
    if (!fn || (ld % 8) != 0 || (reinterpret_cast<uintptr_t>(planes) & 15) != 0) return -1;
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nbatch, 4};
    cuuint64_t strides[3] = {(cuuint64_t)ld * 2, (cuuint64_t)rows * ld * 2, (cuuint64_t)nbatch * rows * ld * 2};
    cuuint32_t box[4] = {tc::BK, tc::BM, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4,
                    const_cast<void*>(planes), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int tc_gemm_launch(const tc::Maps& maps, const tc::Params& p, int grid_m, int grid_n, cudaStream_t s) {
    if (lb_smem_attr((const void*)tc::k_tc_gemm, tc::SMEM_BYTES)) return -1;
    if (grid_m <= 0 || grid_n <= 0 || p.nseg < 1 || p.nseg > tc::MAX_SEGS) return -1;
    if (p.wave < 0)
        for (int g = 0; g < p.nseg; ++g)
            if (p.seg[g].nbatch < 1 || p.seg[g].klen < 1) return -1;
    const int gz = (p.wave < 0 && p.ksplit > 1 && !p.planes) ? p.ksplit : 1;
    tc::k_tc_gemm<<<dim3(grid_m, grid_n, gz), 256, tc::SMEM_BYTES, s>>>(maps, p); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_split_planes(const cplx* X, long long ld_src, int rows, int cols, int transpose, int conj,
                    const double* scale_dev, __half* planes, int ld_dst, long long pstride, int batch,
                    long long src_bstride, long long dst_bstride, cudaStream_t s) {
    // rows_pad: the plane height (dst_bstride / ld_dst); every padded entry is written (zero)
    const int rows_pad = (int)(dst_bstride / ld_dst);
    dim3 grid((ld_dst + 31) / 32, (rows_pad + 31) / 32, batch);
    tc::k_split_planes<<<grid, dim3(32, 8), 0, s>>>(X, ld_src, rows, cols, transpose, conj, scale_dev, planes,
                                                     ld_dst, rows_pad, pstride, src_bstride, dst_bstride); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_split_planes_bf16(const cplx* X, long long ld_src, int rows, int cols, int transpose, void* planes,
                         int ld_dst, long long pstride, cudaStream_t s) {
    const int rows_pad = (int)(pstride / ld_dst);
    dim3 grid((ld_dst + 31) / 32, (rows_pad + 31) / 32, 1);
    tc::k_split_planes_bf16<<<grid, dim3(32, 8), 0, s>>>(X, ld_src, rows, cols, transpose,
                                                          reinterpret_cast<__nv_bfloat16*>(planes), ld_dst, rows_pad,
                                                          pstride); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_maxabs(const cplx* X, long long len, double* part, double* out, cudaStream_t s) {
    constexpr int blocks = 592;
    tc::k_maxabs_part<<<blocks, 256, 0, s>>>(reinterpret_cast<const unsigned long long*>(X), 2 * len,
                                             reinterpret_cast<unsigned long long*>(part)); lb_note_launch();
    tc::k_maxabs_final<<<1, 32, 0, s>>>(reinterpret_cast<const unsigned long long*>(part), blocks, out);
    lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_max_row_l1(const cplx* A, long long rows, int cols, long long ld, double* part, double* out, cudaStream_t s) {
    constexpr int blocks = 592;
    tc::k_row_l1_part<<<blocks, 256, 0, s>>>(A, rows, cols, ld, part); lb_note_launch();
    tc::k_max_part_final<<<1, 32, 0, s>>>(part, blocks, out); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_bound_scale(const double* a, const double* b, const double* c, double* scale_dev, double* inv_dev,
                   double* fac_dev, cudaStream_t s) {
    tc::k_bound_scale<<<1, 32, 0, s>>>(a, b, c, scale_dev, inv_dev, fac_dev); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_pick_scale(const double* maxabs_dev, double* scale_dev, double* inv_dev, cudaStream_t s) {
    tc::k_pick_scale<<<1, 32, 0, s>>>(maxabs_dev, scale_dev, inv_dev); lb_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
