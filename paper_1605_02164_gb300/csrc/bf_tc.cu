// Tensor-core variant of the fused kernel: the Gaussian convolutions of
// Algorithm 1 (the "bulk of the computation" named after Eq. denom) run as
// banded-Toeplitz matrix products on the 5th-generation tensor cores
// (tcgen05.mma, FP16 or BF16 operands, FP32 accumulation in tensor memory).
//
// Per CTA: an output tile of 64 columns x BY rows; its input region (tile
// plus an r-pixel halo, at most 128 x 128 pixels) stays resident in tensor
// memory as FP32 for all K terms.  For each term the region is streamed in
// chunks of 16 rows:
//   A  (all threads) phase theta = 2 pi nu.f in FP32 with range reduction,
//      cos/sin, and the 8 modulated channels cos f_c, cos, sin f_c, sin of
//      16 rows x 128 columns, stored as FP16/BF16 in the K-major operand
//      layout (M = 16 rows x 8 channels = 128, K = columns);
//   M1 (one thread) horizontal pass: 4 output-column blocks of 16, each
//      D1[128 x 16] = A1[128 x Kw] * T[Kw x 16], T the Toeplitz band of the
//      normalised 1-D taps (Kw = 16 + 16 ceil(2r/16));
//   X  (all threads) D1 (TMEM) -> FP16/BF16 into a ring of horizontally
//      blurred rows, laid out MN-major (M = 64 columns x 8 channels);
//   M2 (one thread) vertical pass for the 16 output rows that became
//      complete: 4 M-tiles D2[128 x 16] = A2[128 x Kw] * T[Kw x 16];
//   C  (all threads) combine with the centre pixel's cos/sin into
//      register accumulators P_1..P_3, Z (FP32).
// After the last term out_c = P_c / Z.  Every wait on the tensor core is
// bounded: on timeout the CTA records BF_ERR_TIMEOUT in the status word,
// releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kT = 256;        // threads per CTA (8 warps)
constexpr int kBX = 64;        // output columns per tile
constexpr int kNC = 8;         // 16-row chunks per region (128 rows)
constexpr uint32_t kColF = 0;  // TMEM columns: region f (384), D1 (64), D2 (64)
constexpr uint32_t kColD1 = 384;
constexpr uint32_t kColD2 = 448;
constexpr uint32_t kTmemCols = 512;
constexpr int kSpinLimit = 1 << 22;

struct TcGeom {
    int r, lag, Kw, ksteps, BY, ringC;
    uint32_t offA2, offB, offC;
    uint32_t smem;
};

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets between 8x16-byte
// core matrices, version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B FP16 (0) or
// BF16 (1), A major-ness (0 K-major, 1 MN-major), B K-major, M = 128, N = 16.
__device__ __forceinline__ uint32_t idesc(uint32_t ab_fmt, uint32_t a_mn) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | (a_mn << 15) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (int i = 0; i < kSpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t a, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(a));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t a, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(a));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st8(uint32_t a, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(a),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if constexpr (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

template <int NOC, bool BF16>
__global__ void __launch_bounds__(kT, 1)
    mcsf_tc_kernel(const float *__restrict__ in, float *__restrict__ out, int H, int W, int pitch,
                   const float *__restrict__ nu_hi, int K, const uint16_t *__restrict__ taps, TcGeom g,
                   int *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t taddr_s;
    __shared__ int abort_s;

    uint8_t *A1 = sm;                 // [mg 16][kg 16][8 rows][16 B]   K-major
    uint8_t *A2 = sm + g.offA2;       // [kg Kw/8][tile 4][mg 16][8][16 B]  MN-major ring
    uint8_t *Bt = sm + g.offB;        // [kg Kw/8][ng 2][8 n][16 B]  K-major Toeplitz band
    float2 *ring = reinterpret_cast<float2 *>(sm + g.offC);  // [ringC][64] centre (cos, sin)

    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31, q = w & 3, h = w >> 2;
    const int r = g.r, BY = g.BY;
    const int tx0 = blockIdx.x * kBX, ty0 = blockIdx.y * BY;
    const int rx0 = tx0 - r, ry0 = ty0 - r;
    const size_t plane = (size_t)H * pitch;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;

    // ---- set-up: tensor memory, barriers, Toeplitz band ------------------------
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    for (int i = tid; i < g.Kw * 16; i += kT) {
        const int k = i >> 4, n = i & 15, u = k - n;
        const uint16_t v = (u >= 0 && u <= 2 * r) ? taps[u] : (uint16_t)0;
        *reinterpret_cast<uint16_t *>(Bt + ((k >> 3) * 2 + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2) = v;
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = taddr_s;

    // ---- region f -> tensor memory (FP32, resident for all terms) -------------
    // thread (w, l) owns region row 16c + (l & 15), columns 8 xg .. 8 xg + 7
    // with xg = 2w + (l >> 4), stored in its own TMEM lane at columns
    // (2c + h) * 24 + ch * 8 + j.
    const int row = l & 15, xg = 2 * w + (l >> 4);
    for (int c = 0; c < kNC; ++c) {
        const int gy = ry0 + 16 * c + row;
        const bool rowv = gy >= 0 && gy < H;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int gx = rx0 + 8 * xg + j;
                v[j] = (rowv && gx >= 0 && gx < W) ? __ldg(in + ch * plane + (size_t)gy * pitch + gx) : 0.f;
            }
            tmem_st8(tmem + lane_base + kColF + (2 * c + h) * 24 + ch * 8, v);
        }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();

    float acc[NOC][16];
#pragma unroll
    for (int o = 0; o < NOC; ++o)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[o][j] = 0.f;

    const uint32_t idA1 = idesc(BF16 ? 1u : 0u, 0u);
    const uint32_t idA2 = idesc(BF16 ? 1u : 0u, 1u);
    const uint32_t a1s = smem_u32(A1), a2s = smem_u32(A2), bts = smem_u32(Bt);
    const int kgring = g.Kw >> 3;
    uint32_t ph0 = 0, ph1 = 0;
    bool timed_out = false;

    for (int k = 0; k < K; ++k) {
        const float n0 = __ldg(nu_hi + 3 * k), n1 = __ldg(nu_hi + 3 * k + 1), n2 = __ldg(nu_hi + 3 * k + 2);
        for (int c = 0; c < kNC; ++c) {
            // ---------------- A: cos/sin and modulated channels ----------------
            {
                float f0[8], f1[8], f2[8];
                const uint32_t fa = tmem + lane_base + kColF + (2 * c + h) * 24;
                tmem_ld8(fa, f0);
                tmem_ld8(fa + 8, f1);
                tmem_ld8(fa + 16, f2);
                tmem_wait_ld();
                const int ry = 16 * c + row, gy = ry0 + ry;
                const bool rowv = gy >= 0 && gy < H;
                float cs[8], sn[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int gx = rx0 + 8 * xg + j;
                    const bool v = rowv && gx >= 0 && gx < W;
                    const float t = fmaf(n0, f0[j], fmaf(n1, f1[j], n2 * f2[j]));
                    const float fr = t - rintf(t);
                    float s_, c_;
                    __sincosf(6.28318530717958647692f * fr, &s_, &c_);
                    cs[j] = v ? c_ : 0.f;
                    sn[j] = v ? s_ : 0.f;
                }
                uint8_t *dst = A1 + (size_t)(xg * 128 + (row & 7) * 16);
                const int mg0 = row >> 3;  // + 2 * ch
                uint4 pk;
#define BF_STORE_CH(CH, EXPR)                                                                             \
    {                                                                                                     \
        uint32_t u[4];                                                                                    \
        _Pragma("unroll") for (int p = 0; p < 4; ++p) {                                                   \
            const int j = 2 * p;                                                                          \
            float e0, e1;                                                                                 \
            {                                                                                             \
                const int jj = j;                                                                         \
                e0 = (EXPR);                                                                              \
            }                                                                                             \
            {                                                                                             \
                const int jj = j + 1;                                                                     \
                e1 = (EXPR);                                                                              \
            }                                                                                             \
            u[p] = pack2<BF16>(e0, e1);                                                                   \
        }                                                                                                 \
        pk = make_uint4(u[0], u[1], u[2], u[3]);                                                          \
        *reinterpret_cast<uint4 *>(dst + (size_t)((2 * (CH) + mg0) * 16) * 128) = pk;                     \
    }
                BF_STORE_CH(0, cs[jj] * f0[jj]);
                BF_STORE_CH(1, cs[jj] * f1[jj]);
                BF_STORE_CH(2, cs[jj] * f2[jj]);
                BF_STORE_CH(3, cs[jj]);
                BF_STORE_CH(4, sn[jj] * f0[jj]);
                BF_STORE_CH(5, sn[jj] * f1[jj]);
                BF_STORE_CH(6, sn[jj] * f2[jj]);
                BF_STORE_CH(7, sn[jj]);
#undef BF_STORE_CH
                // centre cos/sin of output pixels, kept for the combine
                if (ry >= r && ry < r + BY) {
                    float2 *rrow = ring + (size_t)(ry % g.ringC) * kBX;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int cx = 8 * xg + j - r;
                        if (cx >= 0 && cx < kBX) rrow[cx] = make_float2(cs[j], sn[j]);
                    }
                }
            }
            fence_async_smem();
            __syncthreads();
            if (abort_s) goto cleanup;
            // ---------------- M1: horizontal pass ------------------------------
            if (tid == 0) {
                fence_after();
#pragma unroll 1
                for (int nc = 0; nc < 4; ++nc)
#pragma unroll 1
                    for (int ks = 0; ks < g.ksteps; ++ks)
                        mma_f16(tmem + kColD1 + 16 * nc, sdesc(a1s + 2 * (nc + ks) * 128, 128, 2048),
                                sdesc(bts + ks * 512, 256, 128), idA1, ks > 0);
                mma_commit(&mbar[0]);
            }
            if (!mbar_wait(&mbar[0], ph0)) timed_out = true;
            ph0 ^= 1;
            fence_after();
            // ---------------- X: D1 -> ring of blurred rows --------------------
            {
                float v[32];
                const uint32_t da = tmem + lane_base + kColD1 + 32 * h;
                tmem_ld16(da, v);
                tmem_ld16(da + 16, v + 16);
                tmem_wait_ld();
                const int ch = 2 * q + (l >> 4), gsel = ch >> 2, p = ch & 3;
                const int kr = (16 * c + row) % g.Kw;
                uint8_t *base = A2 + (size_t)(kr >> 3) * 8192 + (2 * h + gsel) * 2048 + (kr & 7) * 16;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    uint4 pk = make_uint4(pack2<BF16>(v[8 * i], v[8 * i + 1]), pack2<BF16>(v[8 * i + 2], v[8 * i + 3]),
                                          pack2<BF16>(v[8 * i + 4], v[8 * i + 5]),
                                          pack2<BF16>(v[8 * i + 6], v[8 * i + 7]));
                    *reinterpret_cast<uint4 *>(base + (p * 4 + i) * 128) = pk;
                }
            }
            fence_before();
            fence_async_smem();
            if (timed_out) abort_s = 1;
            __syncthreads();
            if (abort_s) goto cleanup;
            // ---------------- M2 + C: vertical pass and combine ----------------
            {
                const int oc = c - g.lag;
                if (oc >= 0 && oc < NOC && 16 * oc < BY) {
                    if (tid == 0) {
                        fence_after();
#pragma unroll 1
                        for (int t = 0; t < 4; ++t)
#pragma unroll 1
                            for (int ks = 0; ks < g.ksteps; ++ks) {
                                const int kg0 = (2 * oc + 2 * ks) % kgring;
                                mma_f16(tmem + kColD2 + 16 * t, sdesc(a2s + kg0 * 8192 + t * 2048, 8192, 128),
                                        sdesc(bts + ks * 512, 256, 128), idA2, ks > 0);
                            }
                        mma_commit(&mbar[1]);
                    }
                    if (!mbar_wait(&mbar[1], ph1)) timed_out = true;
                    ph1 ^= 1;
                    fence_after();
                    float vc[16], vs[16];
                    tmem_ld16(tmem + lane_base + kColD2 + 16 * (2 * h), vc);
                    tmem_ld16(tmem + lane_base + kColD2 + 16 * (2 * h + 1), vs);
                    tmem_wait_ld();
                    const int x = 32 * h + l;
#pragma unroll
                    for (int o = 0; o < NOC; ++o) {
                        if (o == oc) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float2 cs = ring[(size_t)((16 * o + j + r) % g.ringC) * kBX + x];
                                acc[o][j] = fmaf(cs.x, vc[j], fmaf(cs.y, vs[j], acc[o][j]));
                            }
                        }
                    }
                    fence_before();
                    if (timed_out) abort_s = 1;
                }
            }
        }
        __syncthreads();  // term boundary: centre ring rows are reused from row 0
        if (abort_s) goto cleanup;
    }

    // ---- P / Z ----------------------------------------------------------------
    {
        float *zbuf = reinterpret_cast<float *>(sm + g.offC);  // [BY][64], reuses the centre ring
        const int x = 32 * h + l;
        if (q == 3) {
#pragma unroll
            for (int o = 0; o < NOC; ++o)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (16 * o + j < BY) zbuf[(16 * o + j) * kBX + x] = acc[o][j];
        }
        __syncthreads();
        const int gx = tx0 + x;
        if (q < 3 && gx < W) {
#pragma unroll
            for (int o = 0; o < NOC; ++o)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int y = 16 * o + j, gy = ty0 + y;
                    if (y < BY && gy < H) out[q * plane + (size_t)gy * pitch + gx] = acc[o][j] / zbuf[y * kBX + x];
                }
        }
    }

cleanup:
    if (abort_s && tid == 0) {
        atomicCAS(status, 0, BF_ERR_TIMEOUT);
        // drain: wait (bounded) for every MMA issued by this thread
        mma_commit(&mbar[0]);
        mbar_wait(&mbar[0], ph0);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int NOC, bool BF16>
int launch_noc(const float *in, float *out, int H, int W, int pitch, const bf_plan_s &p, const TcGeom &g,
               cudaStream_t s) {
    auto kern = mcsf_tc_kernel<NOC, BF16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem) != cudaSuccess)
        return BF_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    int *st = status_word(dev);
    if (!st) return BF_ERR_NOMEM;
    dim3 grid(cdiv(W, kBX), cdiv(H, g.BY));
    kern<<<grid, kT, g.smem, s>>>(in, out, H, W, pitch, p.nu_hi, p.K, BF16 ? p.tapsbf : p.taps16, g, st);
    return cuda_err(cudaGetLastError());
}

}  // namespace

int launch_tc(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, int variant,
              cudaStream_t s) {
    if (p.d != 3) return BF_ERR_UNSUPPORTED;
    TcGeom g{};
    g.r = p.r;
    g.lag = cdiv(2 * p.r, 16);
    g.Kw = 16 * (g.lag + 1);
    g.ksteps = g.Kw / 16;
    if (48 + g.Kw > 128) return BF_ERR_UNSUPPORTED;
    int noc = (128 - 2 * p.r) / 16;
    if (noc > kNC - g.lag) noc = kNC - g.lag;
    if (noc > 6) noc = 6;
    if (noc < 4) return BF_ERR_UNSUPPORTED;
    g.BY = 16 * noc;
    g.ringC = 16 * (g.lag + 2);
    g.offA2 = 32768;
    g.offB = g.offA2 + (uint32_t)(g.Kw / 8) * 8192;
    g.offC = g.offB + (uint32_t)g.Kw * 32;
    g.offC = (g.offC + 127) & ~127u;
    const uint32_t ring_bytes = (uint32_t)g.ringC * kBX * 8;
    const uint32_t z_bytes = (uint32_t)g.BY * kBX * 4;
    g.smem = g.offC + (ring_bytes > z_bytes ? ring_bytes : z_bytes);
    if (g.smem < 120 * 1024) g.smem = 120 * 1024;  // one CTA per SM: it holds all 512 TMEM columns
    const bool bf = variant == BF_BF16TC;
    switch (noc) {
        case 4: return bf ? launch_noc<4, true>(in, out, H, W, pitch, p, g, s) : launch_noc<4, false>(in, out, H, W, pitch, p, g, s);
        case 5: return bf ? launch_noc<5, true>(in, out, H, W, pitch, p, g, s) : launch_noc<5, false>(in, out, H, W, pitch, p, g, s);
        case 6: return bf ? launch_noc<6, true>(in, out, H, W, pitch, p, g, s) : launch_noc<6, false>(in, out, H, W, pitch, p, g, s);
        default: return BF_ERR_UNSUPPORTED;
    }
}

}  // namespace bf
