// Tensor-core variant of the fused kernel: the Gaussian convolutions of
// Algorithm 1 (the "bulk of the computation" named after Eq. denom) run as
// banded-Toeplitz matrix products on the 5th-generation tensor cores
// (tcgen05.mma, FP16 or BF16 operands, FP32 accumulation in tensor memory).
//
// Per CTA: an output tile of 64 columns x BY rows; its input region (tile
// plus an r-pixel halo, at most 128 x 128 pixels) stays resident in tensor
// memory as FP32 for all K terms.  For each term the region is streamed in
// chunks of 16 rows:
//   A  (compute warps) phase t = nu.f in FP32 turns, reduced to [-1/2, 1/2] by
//      t - rint(t), SFU cos/sin of 2 pi t,
//      and the 8 modulated channels cos f_c, cos, sin f_c, sin of 16 rows x
//      128 columns, stored as FP16/BF16 in the K-major operand layout
//      (M = 16 rows x 8 channels = 128, K = columns);
//   M1 (one issuer thread) horizontal pass, one chain of m128n64k16 MMAs:
//      D1[128 x 64] = A1[128 x Kw1] * T1[Kw1 x 64], T1 the Toeplitz band of
//      the normalised 1-D taps (Kw1 = 16 ceil((64 + 2r) / 16));
//   X  (compute warps) D1 (TMEM) -> FP16/BF16 into a ring of horizontally
//      blurred rows, laid out MN-major (M = 64 columns x 8 channels);
//   M2 (4 issuer threads) vertical pass for the 16 output rows that became
//      complete: 4 M-tiles D2[128 x 16] = A2[128 x Kw] * T2[Kw x 16]
//      (Kw = 16 + 16 ceil(2r / 16));
//   C  (compute warps) combine with the centre pixel's cos/sin into
//      register accumulators P_1..P_3, Z (FP32).
// After the last term out_c = P_c / Z.  Every wait on the tensor core is
// bounded: on timeout the CTA records BF_ERR_TIMEOUT in the status word,
// releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kComputeWarps = 16;  // channels, transpose, combine
constexpr int kComputeThreads = 32 * kComputeWarps;
constexpr int kT = kComputeThreads + 128;  // + one warpgroup that issues the MMAs
// Registers per thread: the launch gives every thread kRegsLaunch (ptxas, from
// the launch bounds); the issuer warpgroup then drops to kRegsIssuer and the
// compute warps rise to kRegsCompute.  The shares must fit in the launch's total.
constexpr int kRegsLaunch = 96, kRegsIssuer = 32, kRegsCompute = 112;
static_assert(128 * kRegsIssuer + kComputeThreads * kRegsCompute <= kT * kRegsLaunch, "register split");
constexpr int kBX = 64;        // output columns per tile
constexpr int kNC = 8;         // 16-row chunks per region (128 rows)
constexpr int kNOC = 5;        // output chunks (of 16 rows) per tile at most
constexpr int kNOC6 = 4;       // the same for six-channel images
constexpr uint32_t kColF = 0;  // TMEM columns: region f (384), D1 (64), D2 (64)
constexpr uint32_t kColD1 = 384;
constexpr uint32_t kColD2 = 448;
constexpr uint32_t kTmemCols = 512;
constexpr int kSpinLimit = 1 << 22;
constexpr int kInjectSpin = 1 << 12;  // spin limit of a launch with BF_FAULT_TC_WAIT armed
// Centre ring: float2 (cos, sin) per output column; ring row t holds flat output
// row t mod ringC, ringC = 16 (lag + 3) (flat output row = flat region row - r).
// Column c of ring row t is stored at t * kBX + (c ^ ring_xor(t)): whatever r,
// the 16 rows a half-warp writes (rows 8-15 four pixels to the side of rows 0-7,
// see px0) and the 32 columns a warp reads in one row fall on distinct banks.
// A combine reads 8 rows starting at a multiple of 8, so its XORs are constants.
__host__ __device__ constexpr int ring_xor(int t) { return (t & 3) | ((t & 4) << 1); }

// Geometries with a specialised step loop in the kernel (the dispatch on
// TcImg::spec lists the same values): the default tile of the lag classes
// r = 1..8, 9..16 and 17..24; the 32-row tiles a 512 x 512 image takes alone at
// r = 1..8 and 9..16 (two-term centre ring); the 64-row tile of a 1024 x 1024
// image alone at r = 9..16; for six-channel images, whose tiles are at most
// 64 rows, also the 64-row tiles of r = 1..8, 17..24 and 25..32 (dmask: bit 0
// three-channel, bit 1 six-channel images).  (A three-channel tile of r =
// 25..32 keeps the general loop: its 128-row centre ring would take the
// shared memory past 227 KB.)
constexpr int kNumSpec = 9;
struct SpecGeom {
    int nc, lag, BY, terms, dmask;
};
constexpr SpecGeom kSpecGeom[kNumSpec] = {{6, 1, 80, 1, 1}, {7, 2, 80, 1, 1}, {8, 3, 80, 1, 1},
                                          {3, 1, 32, 2, 3}, {4, 2, 32, 2, 3}, {6, 2, 64, 1, 3},
                                          {5, 1, 64, 1, 2}, {7, 3, 64, 1, 2}, {8, 4, 64, 1, 2}};
template <int V>
using IC = std::integral_constant<int, V>;

// One image of a launch (the single-image call is a batch of one).  The table
// lives in device memory; tiles of all images form one work queue.
struct TcImg {
    const float *in;
    float *out;
    const float *nu_hi;     // K x 3 frequencies (turns), FP32
    const uint16_t *taps;   // FP16 or BF16 bits of the normalised 1-D taps
    int H, W, pitch, K;
    int r, lag;
    int Kw, ksteps;         // vertical pass: window rows 16 (lag + 1), K-steps of 16
    int Kw1, ks1;           // horizontal pass: 64 + 2r rounded up to 16, K-steps of 16
    int BY, nc, ringC;      // output rows per tile, 16-row chunks per term, centre-ring rows
    int tiles_x, tile_begin, ringA;  // ringA: rows of the blurred-row ring
    int spec, d;                     // spec: index + 1 into kSpecGeom, or 0 (general loop); d = 3 or 6
    // d = 6: the image's per-channel range as order keys (minima at mm[0..5],
    // maxima at mm[6 n_imgs + 0..5]), written by tc_range_kernel before the launch
    uint32_t *mm;
};
static_assert(sizeof(TcImg) == 112, "descriptor layout");

// Shared-memory layout of a launch, sized for the largest window in it.
struct TcLayout {
    uint32_t offA2, offB1, offB, offC, smem;
    int fix;     // the specialised loop every image of the launch runs (kSpecGeom index + 1), or 0
    int spin;    // try_wait attempts before a wait on the tensor core gives up
    int inject;  // 1: skip the first MMA group of every tile (BF_FAULT_TC_WAIT), so the wait runs out
    int d6;      // 1: the launch's images have six channels (the D6 kernel)
};



// Launch control words kept in device scratch: [0] tile counter (zeroed by
// the copy that uploads the image table before every launch).
constexpr int kCtrlWords = 64;  // 256 bytes, so the descriptor table after it stays 256-byte aligned

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
// BF16 (1), A major-ness (0 K-major, 1 MN-major), B K-major, M = 128, N.
__device__ __forceinline__ uint32_t idesc(uint32_t ab_fmt, uint32_t a_mn, uint32_t n) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | (a_mn << 15) | ((n >> 3) << 17) | ((128u >> 4) << 24);
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

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int limit) {
    const uint32_t a = smem_u32(bar);
    for (int i = 0; i < limit; ++i) {
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

// Barrier of the compute warps only (named barrier 1); returns whether any of
// them passed `v` true, so that all take the same branch after it.
__device__ __forceinline__ bool compute_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kComputeThreads)
        : "memory");
    return r != 0;
}

// Step barrier (named barrier 2, all kT threads): the compute warps arrive
// without waiting, the issuer warps wait in hardware (no polling).
__device__ __forceinline__ void step_arrive() { asm volatile("bar.arrive 2, %0;" ::"n"(kT) : "memory"); }
__device__ __forceinline__ void step_wait() { asm volatile("bar.sync 2, %0;" ::"n"(kT) : "memory"); }

// Index checks of the checked build (BF_DEVICE_CHECKS): a failed check records
// BF_ERR_BOUNDS in the status word and the access it guards is skipped.  In the
// normal build the check is the constant true and compiles away.
#ifdef BF_DEVICE_CHECKS
__device__ __forceinline__ bool dcheck(bool ok, int *status) {
    if (!ok) atomicCAS(status, 0, BF_ERR_BOUNDS);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool dcheck(bool, int *) { return true; }
#endif

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld4(uint32_t a, float *v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st4(uint32_t a, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(__float_as_uint(v[0])),
                 "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8u(uint32_t a, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(a));
}

__device__ __forceinline__ void tmem_ld4u(uint32_t a, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void tmem_st8u(uint32_t a, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(a), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st4u(uint32_t a, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]),
                 "r"(v[3])
                 : "memory");
}

// Six-channel region codes: a float's bits mapped to an unsigned key with the
// same order (for the block-wide min / max), and the 16-bit affine code
// f ~ lo + scale * code, decoded as (2^23 + code) * scale + (lo - 2^23 scale)
// in one FMA (absolute error <= scale).
__device__ __forceinline__ uint32_t order_key(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_unkey(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
__device__ __forceinline__ float decode16(uint32_t code, float scale, float c0) {
    return fmaf(__uint_as_float(0x4B000000u | code), scale, c0);
}

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

// Element-pair packing and products for the FP16 / BF16 operands.
template <bool BF16>
struct Pair;
template <>
struct Pair<false> {
    using T = __half2;
    static __device__ __forceinline__ T make(float a, float b) { return __floats2half2_rn(a, b); }
};
template <>
struct Pair<true> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ T make(float a, float b) { return __floats2bfloat162_rn(a, b); }
};
template <typename T>
__device__ __forceinline__ uint32_t bits(T v) {
    static_assert(sizeof(T) == 4, "packed pair");
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

// Persistent kernel, warp-specialised.  Warps 0-15 do the CUDA-core work
// (channels, D1 -> ring, combine); warps 16-19 only issue MMAs.  A
// tcgen05.mma holds its issuing thread until the tensor pipe takes it, so an
// issuer spends most of the pipe's time for a step waiting (~1000 cycles at
// r = 24); on warps of their own those waits no longer hold up the step's
// CUDA-core work.  The issuer warpgroup gives up registers (setmaxnreg) so
// that the compute warps keep kRegsCompute.
// Each CTA keeps its tensor memory and pops tiles (of all images) from a
// device work counter until the queue is empty.  Per tile, a software
// pipeline over the flat sequence of (term, 16-row chunk) steps
// s = k * nc + c.  The compute warps in step s
//   1  build the channels of chunk s+1 (A) into the A1 buffer not being read,
//   1b wait for the vertical MMAs issued after step s-1 and combine them (C),
//   2  wait for the horizontal MMAs of chunk s and move D1 into the ring (X),
//   3  meet at a compute-only barrier and arrive on the step barrier;
// then the issuer warps issue, when chunk s completes 16 output rows, the 4
// vertical M-tiles (one chain of N = 16, K = 16 + 16 ceil(2r/16) per warp),
// and the horizontal MMAs of chunk s+1 (one chain of N = 64, K = 64 + 2r,
// warp 16).  Each MMA group runs while the compute warps do a step of work.
// TMEM: region f 0..383, D1 384..447, D2 448..511 (single-buffered: each is
// read back before the group that rewrites it is issued).
// FIX = 0 chooses each tile's step loop from its image (TcImg::spec); FIX = j
// compiles in only loop j, for a launch whose images all have that geometry.
// Measured on GB300: the kernel with loop 4 or 5 alone (the two-term rings of
// a 512 x 512 image) is 4 % faster than the dispatching one, while for loops 1,
// 2, 3 and 6 the dispatching kernel is ~1 % faster (ptxas arranges the two
// differently), so only FIX = 4 and 5 are built.
// D6 = true: the kernel for six-channel images.  Each term runs as two passes
// of 8 channels in the layout of the three-channel kernel (cos f_1..f_4 and
// sin f_1..f_4; then cos f_5, cos f_6, cos, 0 and sin f_5, sin f_6, sin, 0);
// the region is held as 16-bit codes of a per-tile, per-channel affine map
// (6 channels x 128 columns fit the same 384 TMEM columns), tiles are at most
// 64 rows (two sets of accumulators), and every tile runs the general loop.
template <bool BF16, int FIX, bool D6>
__global__ void __launch_bounds__(kT, 1)
    mcsf_tc_kernel(const TcImg *__restrict__ imgs, int n_imgs, int total_tiles, int *__restrict__ ctrl,
                   int *__restrict__ status, TcLayout lay) {
    constexpr int NOC = D6 ? kNOC6 : kNOC;
    constexpr int NP = D6 ? 2 : 1;  // passes per term
    using P2 = Pair<BF16>;
    extern __shared__ __align__(1024) uint8_t sm[];
    // [0] horizontal MMAs done, [1] vertical MMAs done (4 issuers), [2..5]
    // drain barrier of each issuer warp
    __shared__ __align__(8) uint64_t mbar[6];
    __shared__ uint32_t taddr_s;
    __shared__ int tile_s, cstop_s;
    // six-channel tiles: the image's minimum keys, then scale[0..5], -, -, c0[0..5], -, - of the affine codes
    __shared__ uint32_t mm_s[6];
    __shared__ __align__(16) float aff_s[16];

    uint8_t *A1 = sm;               // 2 x [mg 16][kg 16][8 rows][16 B]   K-major (double buffer)
    uint8_t *A2 = sm + lay.offA2;   // [kg ringA/8][tile 4][mg 16][8][16 B]  MN-major ring of blurred rows
    uint8_t *B1 = sm + lay.offB1;   // [kg Kw1/8][ng 8][8 n][16 B]  K-major band, horizontal pass (N = 64)
    uint8_t *B2 = sm + lay.offB;    // [kg Kw/8][ng 2][8 n][16 B]   K-major band, vertical pass (N = 16)
    float2 *ring = reinterpret_cast<float2 *>(sm + lay.offC);  // [ringC][64] centre (cos, sin), see ring_xor
    int *counter = ctrl;

    // Compute warp w works on TMEM lane quarter q = w & 3 (the lanes it may
    // access), x half h, and half e of the 8-pixel groups / of the 16 rows of a block.
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31, q = w & 3, h = (w >> 2) & 1, e = (w >> 3) & 1;
    const bool issuer = w >= kComputeWarps;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    // The thread owns pixels px0 .. px0 + 3 of its 8-pixel group; rows 8-15 take
    // the other half than rows 0-7 so that the 8-byte stores of a half-warp into
    // a core-matrix row cover all 32 banks.  In TMEM the thread's four pixels sit
    // at the warp-uniform columns pc0 .. pc0 + 3.
    const int row = l & 15, xg = 2 * (w & 7) + (l >> 4), pc0 = 4 * e, px0 = 4 * (e ^ (row >> 3));

    // ---- once per CTA: tensor memory, barriers ------------------------------------
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&mbar[1])) : "memory");  // 4 issuers
        for (int i = 2; i < 6; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        cstop_s = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = taddr_s;
    bool aborted = false;  // every thread, after a barrier that agreed on it
    // Each role runs its own tile loop, so that all of its code comes after its
    // register change.  The barriers of the two loops pair up one to one: tile
    // start; per step, the step barrier (compute -> issuers; when the compute
    // warps stop they arrive once more with cstop_s set); the tile barrier, which
    // also agrees on a stop; z buffer; tile end; final.
    if (issuer) {
        // 4 issuer warps x kRegsIssuer + 16 compute warps x kRegsCompute fit in
        // the 20 x kRegsLaunch the block was launched with.
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsIssuer));
        for (;;) {
            bool iss_stop = false;  // the compute warps stopped
            __syncthreads();        // tile start (tile_s written by thread 0)
            const int tile = tile_s;
            if (tile >= total_tiles) break;
            int im = 0;
            while (im + 1 < n_imgs && __ldg(&imgs[im + 1].tile_begin) <= tile) ++im;
            const TcImg &gg = imgs[im];
            const int K = gg.K, NCr = gg.nc, lag = gg.lag, BY = gg.BY;
            const int S = NP * K * NCr;
            // ---- MMA issue --------------------------------------------------------------
            const int ks1 = gg.ks1, ksteps = gg.ksteps, kgring = gg.ringA >> 3;
            const uint64_t dA1 = sdesc(smem_u32(A1), 128, 2048);  // K-major: LBO = next K group, SBO = next 8 rows
            const uint64_t dB1 = sdesc(smem_u32(B1), 1024, 128);
            const uint64_t dA2 = sdesc(smem_u32(A2), 8192, 128);  // MN-major: LBO = next K group, SBO = next 8 columns
            const uint64_t dB2 = sdesc(smem_u32(B2), 256, 128);
            const int t = w - kComputeWarps;  // vertical M-tile of this warp
            // Descriptors are built per tile; operand offsets are added to the
            // 14-bit start-address field (address >> 4).
            auto issue_M1 = [&](int s) {
                const uint64_t a = dA1 + (uint64_t)((s & 1) * (32768 >> 4));
                const uint32_t id1 = idesc(BF16 ? 1u : 0u, 0u, 64u);
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    if (ks < ks1) mma_f16(tmem + kColD1, a + 16 * ks, dB1 + 128 * ks, id1, ks > 0);
                mma_commit(&mbar[0]);
            };
            auto issue_M2 = [&](int s_first) {
                const uint32_t id2 = idesc(BF16 ? 1u : 0u, 1u, 16u);
                const int kgb = (2 * s_first) % kgring;
#pragma unroll
                for (int ks = 0; ks < 5; ++ks)
                    if (ks < ksteps) {
                        int kg0 = kgb + 2 * ks;
                        if (kg0 >= kgring) kg0 -= kgring;
                        if (!dcheck(kg0 >= 0 && kg0 + 2 <= kgring, status)) continue;
                        mma_f16(tmem + kColD2 + 16 * t, dA2 + (uint64_t)((kg0 * 8192 + t * 2048) >> 4),
                                dB2 + 32 * ks, id2, ks > 0);
                    }
                mma_commit(&mbar[1]);
            };
            // prologue: chunk 0's channels are in A1[0] once the step barrier completes
            step_wait();
            if (cstop_s) {
                iss_stop = true;
                goto iss_tile_end;
            }
            if (t == 0 && l == 0 && !lay.inject) {
                fence_after();
                issue_M1(0);
            }
            __syncwarp();
            {
                int c = 0;
                for (int s = 0; s < S; ++s) {
                    const int oc = c - lag;
                    const bool do_m2 = oc >= 0 && oc < NOC && 16 * oc < BY;
                    step_wait();
                    if (cstop_s) {
                        iss_stop = true;
                        goto iss_tile_end;
                    }
                    if (l == 0) {
                        fence_after();
                        if (do_m2) issue_M2(s - lag);  // needed first: the combine comes before D1 -> ring
                        if (t == 0 && s + 1 < S) issue_M1(s + 1);
                    }
                    __syncwarp();
                    if (++c == NCr) c = 0;
                }
            }
        iss_tile_end:
            fence_before();
            if (__syncthreads_or(iss_stop)) {  // tile barrier
                aborted = true;
                break;
            }
            __syncthreads();  // z buffer
            fence_before();
            __syncthreads();  // tile end
            fence_after();
        }
        if (aborted && l == 0) {
            if (w == kComputeWarps) atomicCAS(status, 0, BF_ERR_TIMEOUT);
            // drain: bounded wait for every MMA this thread issued (a barrier of its own, fresh phase)
            mma_commit(&mbar[2 + (w - kComputeWarps)]);
            mbar_wait(&mbar[2 + (w - kComputeWarps)], 0, lay.spin);
        }
        fence_before();
        __syncthreads();  // final
        return;
    }

    // ---- compute warps --------------------------------------------------------------------
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsCompute));
    const uint16_t *band_taps = nullptr;  // the taps the Toeplitz bands in smem were built from
    uint32_t ph1 = 0, ph2 = 0;  // phases of mbar[0], mbar[1] (carry over from tile to tile)
    for (;;) {
        bool timed_out = false;  // a wait on the tensor core ran out
        if (tid == 0) tile_s = atomicAdd(counter, 1);
        __syncthreads();  // tile start
        const int tile = tile_s;
        if (tile >= total_tiles) break;
        int im = 0;
        while (im + 1 < n_imgs && __ldg(&imgs[im + 1].tile_begin) <= tile) ++im;
        const TcImg g = imgs[im];
        const int K = g.K, NCr = g.nc, lag = g.lag, BY = g.BY;
        const int KP = NP * K;  // "terms" of the step sequence: passes
        const int S = KP * NCr;
        const float *__restrict__ in = g.in;
        float *__restrict__ out = g.out;
        const float *__restrict__ nu_hi = g.nu_hi;
        const int H = g.H, W = g.W, pitch = g.pitch, r = g.r;
        const int tl = tile - g.tile_begin;
        const int ty = tl / g.tiles_x, tx = tl - ty * g.tiles_x;
        const int tx0 = tx * kBX, ty0 = ty * BY;
        const int rx0 = tx0 - r, ry0 = ty0 - r;
        const size_t plane = (size_t)H * pitch;

        // Toeplitz bands of the plan's normalised taps, rebuilt whenever the tile's
        // plan differs from the previous tile's (images of one radius r differ
        // in sigma_s, so the taps, not r, identify the bands; uniform across the
        // compute warps)
        if (g.taps != band_taps) {
            for (int i = tid; i < g.Kw1 * 64; i += kComputeThreads) {
                const int k = i >> 6, n = i & 63, u = k - n;
                const uint16_t v = (u >= 0 && u <= 2 * r) ? g.taps[u] : (uint16_t)0;
                *reinterpret_cast<uint16_t *>(B1 + ((k >> 3) * 8 + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2) = v;
            }
            for (int i = tid; i < g.Kw * 16; i += kComputeThreads) {
                const int k = i >> 4, n = i & 15, u = k - n;
                const uint16_t v = (u >= 0 && u <= 2 * r) ? g.taps[u] : (uint16_t)0;
                *reinterpret_cast<uint16_t *>(B2 + ((k >> 3) * 2 + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2) = v;
            }
            band_taps = g.taps;
        }

        // ---- region f -> tensor memory; in-image masks -------------------------------
        // The 8-pixel group (region row 16c + row, columns 8 xg .. 8 xg + 7) of
        // every chunk c lives in TMEM lane 32q + l at columns (2c + h)*24 +
        // ch*8 + pc0 + jj for pixel px0 + jj of this thread.
        uint32_t vmask = 0;  // bit 4c + jj: pixel px0 + jj inside the image
        uint32_t cmask = 0;  // bit jj: column is a centre (output) column
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int cx = 8 * xg + px0 + jj - r;
            if (cx >= 0 && cx < kBX) cmask |= 1u << jj;
        }
        if constexpr (D6) {
            // Six channels as 16-bit codes of an affine map per image and channel,
            // spanning the image's values (f ~ lo + scale code, scale = (max - min)
            // / 65535; the same map for every tile, so results do not depend on
            // the tiling): 4 pixels x 6 channels = 12 words per
            // thread and chunk, words 0-7 at columns 8 gi .. 8 gi + 7 and words
            // 8-11 at 256 + 4 gi .. + 3, gi = 2 (2c + h) + e; word 2 ch + p holds
            // pixels 2p, 2p + 1 of channel ch.
            for (int c = 0; c < kNC; ++c) {
                const int gy = ry0 + 16 * c + row;
                const bool rowv = gy >= 0 && gy < H;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int gx = rx0 + 8 * xg + px0 + jj;
                    if (rowv && gx >= 0 && gx < W) vmask |= 1u << (4 * c + jj);
                }
            }
            if (tid == 0) {
                for (int ch = 0; ch < 6; ++ch) {
                    float lo = order_unkey(__ldcg(g.mm + ch)), hi = order_unkey(__ldcg(g.mm + 6 * n_imgs + ch));
                    if (!(hi >= lo)) lo = hi = 0.f;  // no in-image value (cannot happen for a non-empty image)
                    const float scale = (hi - lo) * (1.f / 65535.f);
                    mm_s[ch] = order_key(lo);
                    aff_s[ch] = scale;
                    aff_s[8 + ch] = fmaf(-8388608.f, scale, lo);
                }
            }
            compute_sync_or(false);
            float lo6[6], inv6[6];
#pragma unroll
            for (int ch = 0; ch < 6; ++ch) {
                const float scale = aff_s[ch];
                lo6[ch] = order_unkey(mm_s[ch]);
                inv6[ch] = scale > 0.f ? 1.f / scale : 0.f;
            }
            for (int c = 0; c < kNC; ++c) {
                uint32_t wd[12];
#pragma unroll
                for (int ch = 0; ch < 6; ++ch) {
                    uint32_t code[4];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const long long gy = ry0 + 16 * c + row, gx = rx0 + 8 * xg + px0 + jj;
                        float q16 = 0.f;
                        if (((vmask >> (4 * c + jj)) & 1) && dcheck(gy >= 0 && gy < H && gx >= 0 && gx < W, status))
                            q16 = rintf((__ldg(in + ch * plane + (size_t)gy * pitch + gx) - lo6[ch]) * inv6[ch]);
                        code[jj] = (uint32_t)fminf(fmaxf(q16, 0.f), 65535.f);
                    }
                    wd[2 * ch] = code[0] | (code[1] << 16);
                    wd[2 * ch + 1] = code[2] | (code[3] << 16);
                }
                const int gi = 2 * (2 * c + h) + e;
                if (dcheck(8 * gi + 8 <= 256 && 256 + 4 * gi + 4 <= (int)kColD1, status)) {
                    tmem_st8u(tmem + lane_base + kColF + 8 * gi, wd);
                    tmem_st4u(tmem + lane_base + kColF + 256 + 4 * gi, wd + 8);
                }
            }
        } else
        for (int c = 0; c < kNC; ++c) {
            const int gy = ry0 + 16 * c + row;
            const bool rowv = gy >= 0 && gy < H;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int gx = rx0 + 8 * xg + px0 + jj;
                if (rowv && gx >= 0 && gx < W) vmask |= 1u << (4 * c + jj);
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float v[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const long long gy = ry0 + 16 * c + row, gx = rx0 + 8 * xg + px0 + jj;
                    v[jj] = ((vmask >> (4 * c + jj)) & 1) && dcheck(gy >= 0 && gy < H && gx >= 0 && gx < W, status)
                                ? __ldg(in + ch * plane + (size_t)gy * pitch + gx)
                                : 0.f;
                }
                if (dcheck((2 * c + h) * 24 + ch * 8 + pc0 + 4 <= (int)kColD1, status))
                    tmem_st4(tmem + lane_base + kColF + (2 * c + h) * 24 + ch * 8 + pc0, v);
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

        float acc[NOC][8];  // rows 16 o + 8 e + j of this thread's (channel, column)
#pragma unroll
        for (int o = 0; o < NOC; ++o)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[o][j] = 0.f;

        uint8_t *const dstA = A1 + xg * 128 + (row & 7) * 16 + (row >> 3) * 2048 + 2 * px0;
        // Ring columns of this thread's 4 pixels: the XOR depends on the ring row
        // only through (row - r) & 7, a constant of the tile.
        const int rx = ring_xor((row - r) & 7), cb = 8 * xg + px0 - r;
        const int rcol0 = cb ^ rx, rcol1 = (cb + 1) ^ rx, rcol2 = (cb + 2) ^ rx, rcol3 = (cb + 3) ^ rx;
        float nr0, nr1, nr2, nr3 = 0.f, nr4 = 0.f, nr5 = 0.f;  // frequency of the current term, turns per unit of f
        auto load_nu = [&](int k) {
            if constexpr (D6) {
                nr0 = __ldg(nu_hi + 6 * k);
                nr1 = __ldg(nu_hi + 6 * k + 1);
                nr2 = __ldg(nu_hi + 6 * k + 2);
                nr3 = __ldg(nu_hi + 6 * k + 3);
                nr4 = __ldg(nu_hi + 6 * k + 4);
                nr5 = __ldg(nu_hi + 6 * k + 5);
            } else {
                nr0 = __ldg(nu_hi + 3 * k);
                nr1 = __ldg(nu_hi + 3 * k + 1);
                nr2 = __ldg(nu_hi + 3 * k + 2);
            }
        };
        int pend_oc = -1, pend_slot = 0, pend_pass = 0;
        // second set of accumulators of a six-channel tile (the pass-2 channels f_5, f_6, 1)
        float acc1[D6 ? NOC : 1][8];
#pragma unroll
        for (int o = 0; o < (D6 ? NOC : 1); ++o)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc1[o][j] = 0.f;

        // A: channels of flat step s (chunk c of the term whose frequency is in
        // nr0..nr2) into A1[s & 1]; slot16 = 16 s mod ringC.
        auto stage_A = [&](int s, int c, int slot16) {
            float f0[4], f1[4], f2[4];
            const uint32_t fa = tmem + lane_base + kColF + (2 * c + h) * 24 + pc0;
            tmem_ld4(fa, f0);
            tmem_ld4(fa + 8, f1);
            tmem_ld4(fa + 16, f2);
            tmem_wait_ld();
            const uint32_t vm = (vmask >> (4 * c)) & 0xFu;
            const int ry = 16 * c + row;
            const bool centre_row = ry >= r && ry < r + BY && cmask;
            uint32_t o[8][2];
            float csv[4], snv[4];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float cv[2], sv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int j = 2 * p + u;
                    // phase in turns, reduced to [-1/2, 1/2] before the SFU sin/cos
                    // (Eq. Ht: theta = 2 pi nu.f), so the SFU argument stays within [-pi, pi]
                    float tt = fmaf(nr0, f0[j], fmaf(nr1, f1[j], nr2 * f2[j]));
                    tt -= rintf(tt);
                    float s_, c_;
                    __sincosf(6.28318530717958647692f * tt, &s_, &c_);
                    const bool v = (vm >> j) & 1u;
                    cv[u] = v ? c_ : 0.f;
                    sv[u] = v ? s_ : 0.f;
                    csv[j] = cv[u];
                    snv[j] = sv[u];
                }
                const typename P2::T hc = P2::make(cv[0], cv[1]);
                const typename P2::T hs = P2::make(sv[0], sv[1]);
                o[3][p] = bits(hc);
                o[7][p] = bits(hs);
                if constexpr (BF16) {
                    // BF16 keeps 8 mantissa bits: form the products in FP32 and round once
                    o[0][p] = bits(P2::make(cv[0] * f0[2 * p], cv[1] * f0[2 * p + 1]));
                    o[1][p] = bits(P2::make(cv[0] * f1[2 * p], cv[1] * f1[2 * p + 1]));
                    o[2][p] = bits(P2::make(cv[0] * f2[2 * p], cv[1] * f2[2 * p + 1]));
                    o[4][p] = bits(P2::make(sv[0] * f0[2 * p], sv[1] * f0[2 * p + 1]));
                    o[5][p] = bits(P2::make(sv[0] * f1[2 * p], sv[1] * f1[2 * p + 1]));
                    o[6][p] = bits(P2::make(sv[0] * f2[2 * p], sv[1] * f2[2 * p + 1]));
                } else {
                    // FP16 (11-bit mantissa): packed half2 products of rounded operands
                    const typename P2::T g0 = P2::make(f0[2 * p], f0[2 * p + 1]);
                    const typename P2::T g1 = P2::make(f1[2 * p], f1[2 * p + 1]);
                    const typename P2::T g2 = P2::make(f2[2 * p], f2[2 * p + 1]);
                    o[0][p] = bits(__hmul2(hc, g0));
                    o[1][p] = bits(__hmul2(hc, g1));
                    o[2][p] = bits(__hmul2(hc, g2));
                    o[4][p] = bits(__hmul2(hs, g0));
                    o[5][p] = bits(__hmul2(hs, g1));
                    o[6][p] = bits(__hmul2(hs, g2));
                }
            }
            if (centre_row && dcheck(slot16 + row - r >= -g.ringC && slot16 + row - r < g.ringC, status)) {
                // centre cos/sin for the combine, ring row = flat output row mod ringC
                int slot = slot16 + row - r;
                if (slot < 0) slot += g.ringC;
                float2 *rrow = ring + slot * kBX;
                if (cmask & 1u) rrow[rcol0] = make_float2(csv[0], snv[0]);
                if (cmask & 2u) rrow[rcol1] = make_float2(csv[1], snv[1]);
                if (cmask & 4u) rrow[rcol2] = make_float2(csv[2], snv[2]);
                if (cmask & 8u) rrow[rcol3] = make_float2(csv[3], snv[3]);
            }
            // 4 pixels of one channel = half px0 / 4 of a 16-byte core-matrix row
            uint8_t *dst = dstA + (s & 1) * 32768;
            if (dcheck(dst >= A1 && dst + 7 * 4096 + 8 <= A1 + 65536, status)) {
#pragma unroll
                for (int ch = 0; ch < 8; ++ch)
                    *reinterpret_cast<uint2 *>(dst + ch * 4096) = make_uint2(o[ch][0], o[ch][1]);
            }
        };

        // A for a six-channel tile: pass 0 builds cos f_1..f_4, sin f_1..f_4, pass
        // 1 cos f_5, cos f_6, cos, 0, sin f_5, sin f_6, sin, 0, in the channel
        // slots of the three-channel layout; the phase uses all six channels.
        auto stage_A6 = [&](int s, int c, int slot16, int pass) {
            float fv[6][4];
            {
                uint32_t wd[12];
                const int gi = 2 * (2 * c + h) + e;
                tmem_ld8u(tmem + lane_base + kColF + 8 * gi, wd);
                tmem_ld4u(tmem + lane_base + kColF + 256 + 4 * gi, wd + 8);
                tmem_wait_ld();
                const float4 sc0 = *reinterpret_cast<const float4 *>(aff_s);
                const float4 sc1 = *reinterpret_cast<const float4 *>(aff_s + 4);
                const float4 cc0 = *reinterpret_cast<const float4 *>(aff_s + 8);
                const float4 cc1 = *reinterpret_cast<const float4 *>(aff_s + 12);
                const float scl[6] = {sc0.x, sc0.y, sc0.z, sc0.w, sc1.x, sc1.y};
                const float cst[6] = {cc0.x, cc0.y, cc0.z, cc0.w, cc1.x, cc1.y};
#pragma unroll
                for (int ch = 0; ch < 6; ++ch) {
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const uint32_t w2 = wd[2 * ch + p];
                        fv[ch][2 * p] = decode16(w2 & 0xFFFFu, scl[ch], cst[ch]);
                        fv[ch][2 * p + 1] = decode16(w2 >> 16, scl[ch], cst[ch]);
                    }
                }
            }
            const uint32_t vm = (vmask >> (4 * c)) & 0xFu;
            const int ry = 16 * c + row;
            const bool centre_row = ry >= r && ry < r + BY && cmask;
            uint32_t o[8][2];
            float csv[4], snv[4];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float cv[2], sv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int j = 2 * p + u;
                    // phase in turns, reduced to [-1/2, 1/2] before the SFU sin/cos (Eq. Ht)
                    float tt = fmaf(nr0, fv[0][j], fmaf(nr1, fv[1][j], fmaf(nr2, fv[2][j],
                                    fmaf(nr3, fv[3][j], fmaf(nr4, fv[4][j], nr5 * fv[5][j])))));
                    tt -= rintf(tt);
                    float s_, c_;
                    __sincosf(6.28318530717958647692f * tt, &s_, &c_);
                    const bool v = (vm >> j) & 1u;
                    cv[u] = v ? c_ : 0.f;
                    sv[u] = v ? s_ : 0.f;
                    csv[j] = cv[u];
                    snv[j] = sv[u];
                }
                const typename P2::T hc = P2::make(cv[0], cv[1]);
                const typename P2::T hs = P2::make(sv[0], sv[1]);
                // channel q of the pass: f_{q+1} (pass 0), f_5, f_6, 1, 0 (pass 1)
                auto prod = [&](int ch, float t0, float t1, typename P2::T ht) -> uint32_t {
                    if constexpr (BF16)
                        return bits(P2::make(t0 * fv[ch][2 * p], t1 * fv[ch][2 * p + 1]));
                    else
                        return bits(__hmul2(ht, P2::make(fv[ch][2 * p], fv[ch][2 * p + 1])));
                };
                if (pass == 0) {
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        o[q4][p] = prod(q4, cv[0], cv[1], hc);
                        o[4 + q4][p] = prod(q4, sv[0], sv[1], hs);
                    }
                } else {
                    o[0][p] = prod(4, cv[0], cv[1], hc);
                    o[1][p] = prod(5, cv[0], cv[1], hc);
                    o[2][p] = bits(hc);
                    o[3][p] = 0u;
                    o[4][p] = prod(4, sv[0], sv[1], hs);
                    o[5][p] = prod(5, sv[0], sv[1], hs);
                    o[6][p] = bits(hs);
                    o[7][p] = 0u;
                }
            }
            if (centre_row && dcheck(slot16 + row - r >= -g.ringC && slot16 + row - r < g.ringC, status)) {
                int slot = slot16 + row - r;
                if (slot < 0) slot += g.ringC;
                float2 *rrow = ring + slot * kBX;
                if (cmask & 1u) rrow[rcol0] = make_float2(csv[0], snv[0]);
                if (cmask & 2u) rrow[rcol1] = make_float2(csv[1], snv[1]);
                if (cmask & 4u) rrow[rcol2] = make_float2(csv[2], snv[2]);
                if (cmask & 8u) rrow[rcol3] = make_float2(csv[3], snv[3]);
            }
            uint8_t *dst = dstA + (s & 1) * 32768;
            if (dcheck(dst >= A1 && dst + 7 * 4096 + 8 <= A1 + 65536, status)) {
#pragma unroll
                for (int ch = 0; ch < 8; ++ch)
                    *reinterpret_cast<uint2 *>(dst + ch * 4096) = make_uint2(o[ch][0], o[ch][1]);
            }
        };

        // C: combine output chunk oc; slot0 = ring row of its output row 16 oc + 8 e
        // (a multiple of 8 at most ringC - 8: the 8 rows read never wrap)
        auto stage_C = [&](int oc, int slot0, int pass = 0) {
            if (!dcheck(slot0 >= 0 && slot0 + 8 <= g.ringC && oc >= 0 && oc < NOC, status)) return;
            float vc[8], vs[8];  // output rows 16 oc + 8 e + j of the cos / sin M-tile
            tmem_ld8(tmem + lane_base + kColD2 + 16 * (2 * h) + 8 * e, vc);
            tmem_ld8(tmem + lane_base + kColD2 + 16 * (2 * h + 1) + 8 * e, vs);
            tmem_wait_ld();
            const int x = 32 * h + l;
            const float2 *rrow = ring + slot0 * kBX;
#pragma unroll
            for (int o = 0; o < NOC; ++o) {
                if (o == oc) {
                    if (D6 && pass) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float2 cs = rrow[j * kBX + (x ^ ring_xor(j))];
                            acc1[D6 ? o : 0][j] = fmaf(cs.x, vc[j], fmaf(cs.y, vs[j], acc1[D6 ? o : 0][j]));
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float2 cs = rrow[j * kBX + (x ^ ring_xor(j))];
                            acc[o][j] = fmaf(cs.x, vc[j], fmaf(cs.y, vs[j], acc[o][j]));
                        }
                    }
                }
            }
        };

        // X: D1 of a flat step -> A2 ring; kr16 = 16 s mod Kw
        auto stage_X = [&](int kr16) {
            float v[16];  // output columns 32 h + 16 e .. + 15 of this (channel, row)
            tmem_ld16(tmem + lane_base + kColD1 + 32 * h + 16 * e, v);
            tmem_wait_ld();
            const int ch = 2 * q + (l >> 4), gsel = ch >> 2, p = ch & 3;
            const int kr = kr16 + row;
            uint8_t *base =
                A2 + (size_t)(kr >> 3) * 8192 + (2 * h + gsel) * 2048 + (kr & 7) * 16 + p * 512 + 2 * e * 128;
            if (!dcheck(kr >= 0 && kr < g.ringA, status)) return;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const uint4 pk = make_uint4(bits(P2::make(v[8 * i], v[8 * i + 1])), bits(P2::make(v[8 * i + 2], v[8 * i + 3])),
                                            bits(P2::make(v[8 * i + 4], v[8 * i + 5])),
                                            bits(P2::make(v[8 * i + 6], v[8 * i + 7])));
                *reinterpret_cast<uint4 *>(base + i * 128) = pk;
            }
        };

        // End of a step: every compute warp has finished the step's smem writes
        // and TMEM reads (compute barrier), then all arrive on the step barrier.
        // If any compute warp timed out, all of them stop together and tell the
        // issuers through cstop_s.
        auto step_done = [&]() -> bool {
            fence_before();
            fence_async_smem();
            const bool stop = compute_sync_or(timed_out);
            if (stop && tid == 0) cstop_s = 1;
            step_arrive();
            return !stop;
        };

        // ---- prologue ------------------------------------------------------------------
        load_nu(0);
        if constexpr (D6)
            stage_A6(0, 0, 0, 0);
        else
            stage_A(0, 0, 0);
        if (!step_done()) goto cmp_tile_end;

        {
            // Step loops.  A tile whose image has one of the geometries in
            // kSpecGeom (g.spec = its index + 1) runs the loop specialised to it:
            // chunks per term NCT, lag LAGT, NOBT output chunks, a centre ring of
            // PT terms x 16 NCT rows; the chunk loop is unrolled and every ring slot
            // and output chunk of a step is a compile-time constant.  Any other tile
            // runs the general loop.  Both return false when the compute warps stop.
            auto spec_loop = [&](auto nct_c, auto lag_c, auto nob_c, auto pt_c) -> bool {
                constexpr int NCT = decltype(nct_c)::value, LAGT = decltype(lag_c)::value;
                constexpr int NOBT = decltype(nob_c)::value, PT = decltype(pt_c)::value;
                // ---- pipeline, specialised geometry -----------------------------------------------
                // Step (k, c): centre-ring slot tb(k) + 16 c, tb(k) = 16 NCT (k mod PT),
                // output chunk c - LAGT; the A1 buffer (k NCT + c) & 1 and the
                // blurred-row ring rows 16 ((k NCT + c) mod (LAGT + 1)) are constants
                // too when NCT is even / a multiple of LAGT + 1, else they are carried
                // from step to step.  The centre-ring rows a step writes (chunk c + 1,
                // or chunk 0 of the next term) never meet the rows it combines (chunk
                // c - 1 - LAGT, or the previous term's last): NCT >= LAGT + 3 keeps them
                // apart in a one-term ring, PT = 2 puts consecutive terms in different halves.
                static_assert((PT == 1 && NCT >= LAGT + 3) || (PT == 2 && NCT >= LAGT + 1), "geometry");
                static_assert(NOBT <= NOC, "geometry");
                constexpr bool kParConst = NCT % 2 == 0, kRingConst = NCT % (LAGT + 1) == 0;
                auto tbase = [&](int kk) { return PT == 2 ? (kk & 1) * 16 * NCT : 0; };
                // A six-channel tile runs 2K passes as the "terms" k of the loop
                // (pass k & 1 of term k >> 1).
                int krS = 0;  // 16 s mod Kw when it is not a constant
                for (int k = 0; k < KP; ++k) {
                    const int kpar = kParConst ? 0 : (k & 1);
                    const int tb = tbase(k);
    #pragma unroll
                    for (int c = 0; c < NCT; ++c) {
                        if (c + 1 < NCT) {
                            if constexpr (D6)
                                stage_A6(kpar + c + 1, c + 1, tb + 16 * (c + 1), k & 1);
                            else
                                stage_A(kpar + c + 1, c + 1, tb + 16 * (c + 1));
                        } else if (k + 1 < KP) {
                            if constexpr (D6) {
                                if (((k + 1) & 1) == 0) load_nu((k + 1) >> 1);
                                stage_A6(kParConst ? 0 : (k + 1) & 1, 0, tbase(k + 1), (k + 1) & 1);
                            } else {
                                load_nu(k + 1);
                                stage_A(kParConst ? 0 : (k + 1) & 1, 0, tbase(k + 1));
                            }
                        }
                        // output chunk completed by the previous step (of term k - 1 when c = 0)
                        const int ocp = (c == 0 ? NCT - 1 : c - 1) - LAGT;
                        if (ocp >= 0 && ocp < NOBT && (c > 0 || k > 0)) {
                            if (!mbar_wait(&mbar[1], ph2, lay.spin)) timed_out = true;
                            ph2 ^= 1;
                            fence_after();
                            stage_C(ocp, (c == 0 ? tbase(k - 1) : tb) + 16 * ocp + 8 * e, (c == 0 ? k - 1 : k) & 1);
                        }
                        if (!mbar_wait(&mbar[0], ph1, lay.spin)) timed_out = true;
                        ph1 ^= 1;
                        fence_after();
                        if constexpr (kRingConst) {
                            stage_X(16 * (c % (LAGT + 1)));
                        } else {
                            stage_X(krS);
                            krS += 16;
                            if (krS == 16 * (LAGT + 1)) krS = 0;
                        }
                        if (!step_done()) return false;
                    }
                }
                if (NCT - 1 - LAGT >= 0 && NCT - 1 - LAGT < NOBT) {
                    if (!mbar_wait(&mbar[1], ph2, lay.spin)) timed_out = true;
                    ph2 ^= 1;
                    fence_after();
                    stage_C(NCT - 1 - LAGT, tbase(KP - 1) + 16 * (NCT - 1 - LAGT) + 8 * e, (KP - 1) & 1);
                }
                return true;
            };
            auto general_loop = [&]() -> bool {
                // ---- pipeline ----------------------------------------------------------------------
                // Step s is chunk c of term k; slotS = 16 s mod ringC and krS = 16 s mod Kw
                // are carried from step to step (no division in the loop), as are the
                // chunk, term and slot of step s + 1 (cA, kA, slotA).
                // A six-channel tile runs 2K passes ("terms" kA of the sequence);
                // pass kA & 1 of term kA >> 1.
                {
                    int c = 0, kA = 0, cA = 0, slotS = 0, krS = 0;
                    for (int s = 0; s < S; ++s) {
                        const int oc = c - lag;
                        const bool do_m2 = oc >= 0 && oc < NOC && 16 * oc < BY;
                        const int passS = D6 ? (kA & 1) : 0;  // pass of step s
                        if (++cA == NCr) {
                            cA = 0;
                            if (++kA < KP) {
                                if (!D6)
                                    load_nu(kA);
                                else if ((kA & 1) == 0)
                                    load_nu(kA >> 1);
                            }
                        }
                        int slotA = slotS + 16;
                        if (slotA >= g.ringC) slotA -= g.ringC;
                        if (s + 1 < S) {
                            if constexpr (D6)
                                stage_A6(s + 1, cA, slotA, kA & 1);
                            else
                                stage_A(s + 1, cA, slotA);
                        }
                        if (pend_oc >= 0) {
                            if (!mbar_wait(&mbar[1], ph2, lay.spin)) timed_out = true;
                            ph2 ^= 1;
                            fence_after();
                            stage_C(pend_oc, pend_slot, pend_pass);
                            pend_oc = -1;
                        }
                        if (!mbar_wait(&mbar[0], ph1, lay.spin)) timed_out = true;
                        ph1 ^= 1;
                        fence_after();
                        stage_X(krS);
                        if (!step_done()) return false;
                        if (do_m2) {
                            pend_oc = oc;
                            pend_pass = passS;
                            // flat output row 16 (s - lag) + 8 e, mod ringC (16 lag < ringC)
                            int sl = slotS - 16 * lag + 8 * e;
                            if (sl < 0) sl += g.ringC;
                            if (sl >= g.ringC) sl -= g.ringC;
                            pend_slot = sl;
                        }
                        c = cA;
                        slotS = slotA;
                        krS += 16;
                        if (krS == g.ringA) krS = 0;
                    }
                }
                if (pend_oc >= 0) {
                    if (!mbar_wait(&mbar[1], ph2, lay.spin)) timed_out = true;
                    ph2 ^= 1;
                    fence_after();
                    stage_C(pend_oc, pend_slot, pend_pass);
                }
                return true;
            };
            bool go;
            if constexpr (D6) {
                switch (g.spec) {  // the entries of kSpecGeom whose dmask has bit 1
                    case 4: go = spec_loop(IC<3>(), IC<1>(), IC<2>(), IC<2>()); break;
                    case 5: go = spec_loop(IC<4>(), IC<2>(), IC<2>(), IC<2>()); break;
                    case 6: go = spec_loop(IC<6>(), IC<2>(), IC<4>(), IC<1>()); break;
                    case 7: go = spec_loop(IC<5>(), IC<1>(), IC<4>(), IC<1>()); break;
                    case 8: go = spec_loop(IC<7>(), IC<3>(), IC<4>(), IC<1>()); break;
                    case 9: go = spec_loop(IC<8>(), IC<4>(), IC<4>(), IC<1>()); break;
                    default: go = general_loop(); break;
                }
            } else switch (FIX ? FIX : g.spec) {
                case 1: go = spec_loop(IC<6>(), IC<1>(), IC<5>(), IC<1>()); break;
                case 2: go = spec_loop(IC<7>(), IC<2>(), IC<5>(), IC<1>()); break;
                case 3: go = spec_loop(IC<8>(), IC<3>(), IC<5>(), IC<1>()); break;
                case 4: go = spec_loop(IC<3>(), IC<1>(), IC<2>(), IC<2>()); break;
                case 5: go = spec_loop(IC<4>(), IC<2>(), IC<2>(), IC<2>()); break;
                case 6: go = spec_loop(IC<6>(), IC<2>(), IC<4>(), IC<1>()); break;
                default: go = general_loop(); break;
            }
            if (!go) goto cmp_tile_end;
        }

        // ---- P / Z ----------------------------------------------------------------
        fence_before();
        if (__syncthreads_or(timed_out)) {  // tile barrier, with the issuers
            aborted = true;
            break;
        }
        {
            float *zbuf = reinterpret_cast<float *>(sm + lay.offC);  // [BY][64], reuses the centre ring
            const int x = 32 * h + l;
            // Z: channel 3 of the (only) pass, or channel 2 of a six-channel tile's second pass
            if (q == (D6 ? 2 : 3)) {
#pragma unroll
                for (int o = 0; o < NOC; ++o)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (16 * o + 8 * e + j < BY && dcheck((16 * o + 8 * e + j + 1) * kBX * 4 <= (int)(lay.smem - lay.offC), status))
                            zbuf[(16 * o + 8 * e + j) * kBX + x] = D6 ? acc1[D6 ? o : 0][j] : acc[o][j];
            }
            __syncthreads();  // z buffer
            const int gx = tx0 + x;
            // P_{q+1} from the first pass's channel q; a six-channel tile's P_5, P_6
            // from the second pass's channels 0, 1
            if (q < (D6 ? 4 : 3) && gx < W) {
#pragma unroll
                for (int o = 0; o < NOC; ++o)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int y = 16 * o + 8 * e + j, gy = ty0 + y;
                        if (y < BY && gy < H && dcheck(gy >= 0 && gx >= 0 && gx < W, status)) {
                            const float zi = zbuf[y * kBX + x];
                            out[q * plane + (size_t)gy * pitch + gx] = acc[o][j] / zi;
                            if (D6 && q < 2) out[(4 + q) * plane + (size_t)gy * pitch + gx] = acc1[D6 ? o : 0][j] / zi;
                        }
                    }
            }
        }
        fence_before();
        __syncthreads();  // tile end: zbuf, ring and TMEM are reused by the next tile
        fence_after();
        continue;
    cmp_tile_end:  // the compute warps stopped inside the step loop (all of them, see step_done)
        fence_before();
        __syncthreads_or(1);  // tile barrier
        aborted = true;
        break;
    }
    fence_before();
    __syncthreads();  // final
    fence_after();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    (void)aborted;
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------

// Per-image geometry for window radius r; false if the tile scheme cannot hold it.
bool tc_geometry(int r, TcImg &g) {
    g.r = r;
    g.lag = cdiv(2 * r, 16);
    g.Kw = 16 * (g.lag + 1);
    g.ringA = g.Kw;
    g.ksteps = g.Kw / 16;
    g.Kw1 = 16 * cdiv(kBX + 2 * r, 16);
    g.ks1 = g.Kw1 / 16;
    if (g.Kw1 > 128 || g.ksteps > 5) return false;
    int noc = (128 - 2 * r) / 16;
    if (noc > kNC - g.lag) noc = kNC - g.lag;
    if (noc > (g.d == 6 ? kNOC6 : kNOC)) noc = g.d == 6 ? kNOC6 : kNOC;
    if (noc < 1) return false;
    g.BY = 16 * noc;
    g.nc = cdiv(g.BY + 2 * r, 16);
    g.ringC = 16 * (g.lag + 3);  // rows written ahead by stage A never reach the rows stage C reads
    return true;
}

TcLayout tc_layout(int max_ringA, int max_Kw, int max_Kw1, int max_ringC, int max_BY) {
    TcLayout L{};
    L.offA2 = 65536;
    L.offB1 = L.offA2 + (uint32_t)(max_ringA / 8) * 8192;
    L.offB = L.offB1 + (uint32_t)max_Kw1 * 128;
    L.offC = (L.offB + (uint32_t)max_Kw * 32 + 127) & ~127u;
    const uint32_t ring_bytes = (uint32_t)max_ringC * kBX * 8;
    const uint32_t z_bytes = (uint32_t)max_BY * kBX * 4;
    L.smem = L.offC + (ring_bytes > z_bytes ? ring_bytes : z_bytes);
    if (L.smem < 120 * 1024) L.smem = 120 * 1024;  // one CTA per SM: it holds all 512 TMEM columns
    L.fix = 0;
    L.spin = kSpinLimit;
    L.inject = 0;
    L.d6 = 0;
    return L;
}

}  // namespace

// Builds the image table (images ordered by per-tile cost, largest first, so
// the dynamic queue ends on cheap tiles), copies it with zeroed control words
// into `scratch`, and launches one persistent grid.  `scratch` must hold
// tc_scratch_bytes(n) bytes and is owned by the caller for the stream.
size_t tc_scratch_bytes(int n) {
    return (size_t)kCtrlWords * sizeof(int) + (size_t)n * (sizeof(TcImg) + 12 * sizeof(uint32_t));
}

namespace {

// Per-channel range of every six-channel image of a launch (the affine map of
// its 16-bit region codes), as order keys: block-wide min / max of the rows
// the block takes, then one atomic per warp.  The keys start at 0xFFFFFFFF
// (minima) and 0 (maxima).
__global__ void __launch_bounds__(256) tc_range_kernel(const TcImg *__restrict__ imgs, int m) {
  for (int im = blockIdx.y; im < m; im += gridDim.y) {  // grid.y is capped at 65535 images
    const TcImg &g = imgs[im];
    const size_t plane = (size_t)g.H * g.pitch;
    float mn[6], mx[6];
#pragma unroll
    for (int ch = 0; ch < 6; ++ch) {
        mn[ch] = __int_as_float(0x7F800000);
        mx[ch] = -mn[ch];
    }
    for (int y = blockIdx.x; y < g.H; y += gridDim.x)
        for (int x = threadIdx.x; x < g.W; x += blockDim.x)
#pragma unroll
            for (int ch = 0; ch < 6; ++ch) {
                const float v = __ldg(g.in + ch * plane + (size_t)y * g.pitch + x);
                mn[ch] = fminf(mn[ch], v);
                mx[ch] = fmaxf(mx[ch], v);
            }
#pragma unroll
    for (int ch = 0; ch < 6; ++ch) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[ch] = fminf(mn[ch], __shfl_xor_sync(0xFFFFFFFFu, mn[ch], o));
            mx[ch] = fmaxf(mx[ch], __shfl_xor_sync(0xFFFFFFFFu, mx[ch], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int ch = 0; ch < 6; ++ch) {
            atomicMin(g.mm + ch, order_key(mn[ch]));
            atomicMax(g.mm + 6 * m + ch, order_key(mx[ch]));
        }
    }
  }
}

// Range keys of a six-channel table at `keys` (6 m minima, then 6 m maxima):
// set the starting values and launch tc_range_kernel.
int tc_ranges(const TcImg *imgs_dev, uint32_t *keys, int m, cudaStream_t s) {
    if (cudaMemsetAsync(keys, 0xFF, (size_t)6 * m * sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(keys + 6 * m, 0, (size_t)6 * m * sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return BF_ERR_CUDA;
    }
    tc_range_kernel<<<dim3(64, std::min(m, 65535)), 256, 0, s>>>(imgs_dev, m);
    return cuda_err(cudaGetLastError());
}

// Descriptor of one image (tile_begin left 0); false if the tile scheme cannot hold it.
int tc_fill(const bf_item &it, int variant, TcImg &g) {
    const bf_plan_s &p = *it.plan;
    if (p.d != 3 && p.d != 6) return BF_ERR_UNSUPPORTED;
    g = TcImg{};
    g.d = p.d;
    if (!tc_geometry(p.r, g)) return BF_ERR_UNSUPPORTED;
    g.in = it.in;
    g.out = it.out;
    g.nu_hi = p.nu_hi;
    g.taps = variant == BF_BF16TC ? p.tapsbf : p.taps16;
    g.H = it.H;
    g.W = it.W;
    g.pitch = it.pitch;
    g.K = p.K;
    g.tiles_x = cdiv(it.W, kBX);
    return BF_OK;
}

// One image alone: the tile height (a multiple of 16 rows, at most the one the
// geometry allows) that minimises (waves of tiles over the SMs) x (16-row steps
// per tile), so that a small image spreads over all SMs.  A pixel's arithmetic
// does not depend on it: tile origins stay multiples of 16 rows.  Batches keep
// the tallest tile; their queue balances the SMs.
// Output rows of a tile: 16 noc, at most what the geometry allows (noc_max).
void tc_set_noc(TcImg &g, int noc, int noc_max) {
    if (noc > noc_max) noc = noc_max;
    if (noc < 1) noc = 1;
    g.BY = 16 * noc;
    g.nc = cdiv(g.BY + 2 * g.r, 16);
}

void tc_fit_waves(TcImg &g) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        return;
    }
    long long best_cost = -1;
    int best = g.BY / 16;
    for (int noc = g.BY / 16; noc >= 1; --noc) {
        const long long tiles = (long long)g.tiles_x * cdiv(g.H, 16 * noc);
        const long long cost = (tiles + nsm - 1) / nsm * cdiv(16 * noc + 2 * g.r, 16);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = noc;
        }
    }
    g.BY = 16 * best;
    g.nc = cdiv(g.BY + 2 * g.r, 16);
}

// Tile offsets, the step loop of each image (kSpecGeom) and the shared-memory
// layout of an ordered table.  An image with a specialised loop has a centre
// ring of 16 nc rows per term of that loop, if that ring fits in the shared
// memory the rest of the launch's layout leaves (a batch that mixes in a wide
// window may not leave it); otherwise it runs the general loop.
void tc_finish(TcImg *tab, int m, int *total, TcLayout *lay) {
    int max_ringA = 16, max_Kw = 16, max_Kw1 = 64, max_ringC = 48, max_BY = 16, t = 0;
    for (int i = 0; i < m; ++i) {
        tab[i].tile_begin = t;
        t += tab[i].tiles_x * cdiv(tab[i].H, tab[i].BY);
        max_ringA = std::max(max_ringA, tab[i].ringA);
        max_Kw = std::max(max_Kw, tab[i].Kw);
        max_Kw1 = std::max(max_Kw1, tab[i].Kw1);
        max_ringC = std::max(max_ringC, tab[i].ringC);  // the general loop's rings
        max_BY = std::max(max_BY, tab[i].BY);
    }
    int dev = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        max_smem = 0;  // no specialised rings
    }
    const TcLayout base = tc_layout(max_ringA, max_Kw, max_Kw1, 0, max_BY);
    const long long ring_rows = ((long long)max_smem - 1024 - (long long)base.offC) / (kBX * 8);
    for (int i = 0; i < m; ++i) {
        tab[i].spec = 0;
        for (int j = 0; j < kNumSpec; ++j) {
            if (!((kSpecGeom[j].dmask >> (tab[i].d == 6 ? 1 : 0)) & 1)) continue;
            const int rows = 16 * kSpecGeom[j].nc * kSpecGeom[j].terms;
            if (tab[i].nc == kSpecGeom[j].nc && tab[i].lag == kSpecGeom[j].lag && tab[i].BY == kSpecGeom[j].BY &&
                rows <= ring_rows) {
                tab[i].spec = j + 1;
                tab[i].ringC = rows;
            }
        }
        max_ringC = std::max(max_ringC, tab[i].ringC);
    }
    *total = t;
    *lay = tc_layout(max_ringA, max_Kw, max_Kw1, max_ringC, max_BY);
    int fix = m > 0 ? tab[0].spec : 0;
    for (int i = 1; i < m; ++i)
        if (tab[i].spec != fix) fix = 0;
    lay->fix = (fix == 4 || fix == 5) ? fix : 0;  // the kernels built with one loop (see FIX)
}

// Launch over a table already in device memory.  The table is ordered by
// per-tile cost (largest first) so the dynamic queue ends on cheap tiles.
int tc_launch(const TcImg *imgs_dev, int m, int total, int *ctrl_dev, int *status_dev, const TcLayout &lay_in,
              int variant, cudaStream_t s) {
    TcLayout lay = lay_in;
    if (take_fault(BF_FAULT_TC_WAIT)) {
        lay.inject = 1;
        lay.spin = kInjectSpin;
    }
    int dev = 0, max_smem = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if ((int)lay.smem + 1024 > max_smem) return BF_ERR_UNSUPPORTED;  // + the 1 KB-aligned static part
    using Kern = void (*)(const TcImg *, int, int, int *, int *, TcLayout);
    Kern kern;
    const bool b = variant == BF_BF16TC;
    if (lay.d6) {
        kern = b ? mcsf_tc_kernel<true, 0, true> : mcsf_tc_kernel<false, 0, true>;
    } else {
        switch (lay.fix) {
            case 0: kern = b ? mcsf_tc_kernel<true, 0, false> : mcsf_tc_kernel<false, 0, false>; break;
            case 4: kern = b ? mcsf_tc_kernel<true, 4, false> : mcsf_tc_kernel<false, 4, false>; break;
            case 5: kern = b ? mcsf_tc_kernel<true, 5, false> : mcsf_tc_kernel<false, 5, false>; break;
            default: return BF_ERR_ARG;
        }
    }
    // The register split inside the kernel assumes the launch gives each thread
    // kRegsLaunch registers; with fewer the compute warps' request could not be met.
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
        cudaGetLastError();
        return BF_ERR_CUDA;
    }
    if (fa.numRegs != kRegsLaunch) return BF_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem) != cudaSuccess) {
        cudaGetLastError();
        return BF_ERR_CUDA;
    }
    kern<<<std::min(total, nsm), kT, lay.smem, s>>>(imgs_dev, m, total, ctrl_dev, status_dev, lay);
    return cuda_err(cudaGetLastError());
}

bool cost_before(const TcImg &a, const TcImg &b) {
    const long long ca = (long long)a.K * a.nc * (a.d == 6 ? 2 : 1), cb = (long long)b.K * b.nc * (b.d == 6 ? 2 : 1);
    if (ca != cb) return ca > cb;
    return a.r < b.r;
}

// Fills, orders and finishes the table of the call's images with d_sel
// channels (3 or 6: one launch each); shared by both batch entry points so
// that they launch identical work (a lone image gets its fitted tile height
// in both).  m = number of non-empty images taken.
int tc_prepare(const bf_item *items, int n, int variant, int d_sel, TcImg *tab, int *m_out, int *total,
               TcLayout *lay) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        if (items[i].H == 0 || items[i].W == 0) continue;
        const int d = items[i].plan->d;
        if (d != 3 && d != 6) return BF_ERR_UNSUPPORTED;
        if (d != d_sel) continue;
        const int rc = tc_fill(items[i], variant, tab[m]);
        if (rc != BF_OK) return rc;
        ++m;
    }
    *m_out = m;
    if (m == 0) return BF_OK;
    // tile height: a measured one from the tuning table, else the cost model
    // (tc_fit_waves alone; the geometry's tallest tile in a batch)
    const int ctx = m == 1 ? BF_TUNE_ALONE : BF_TUNE_BATCH;
    for (int i = 0; i < m; ++i) {
        const int rows = tune_rows(variant, d_sel, tab[i].r, tab[i].H, tab[i].W, ctx);
        if (rows > 0)
            tc_set_noc(tab[i], rows / 16, tab[i].BY / 16);
        else if (m == 1)
            tc_fit_waves(tab[i]);
    }
    for (int a = 1; a < m; ++a) {  // stable insertion sort by cost (no temporary buffer)
        const TcImg t = tab[a];
        int b = a - 1;
        while (b >= 0 && cost_before(t, tab[b])) {
            tab[b + 1] = tab[b];
            --b;
        }
        tab[b + 1] = t;
    }
    tc_finish(tab, m, total, lay);
    lay->d6 = d_sel == 6;
    return BF_OK;
}

}  // namespace

int tc_launch_batch(const bf_item *items, int n, int variant, void *scratch, int *status, cudaStream_t s) {
    if (n <= 0) return BF_OK;
    // One persistent launch for the three-channel images, then one for the
    // six-channel ones, in stream order through the same scratch.
    for (const int d_sel : {3, 6}) {
        std::vector<unsigned char> host(tc_scratch_bytes(n), 0);  // control words (zero) + table
        TcImg *tab = reinterpret_cast<TcImg *>(host.data() + kCtrlWords * sizeof(int));
        int m = 0, total = 0;
        TcLayout lay{};
        int rc = tc_prepare(items, n, variant, d_sel, tab, &m, &total, &lay);
        if (rc != BF_OK) return rc;
        if (m == 0) continue;
        const size_t bytes = (size_t)kCtrlWords * sizeof(int) + (size_t)m * sizeof(TcImg);
        uint32_t *keys = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(scratch) + bytes);
        for (int i = 0; i < m; ++i) tab[i].mm = d_sel == 6 ? keys + 6 * i : nullptr;
        if (cudaMemcpyAsync(scratch, host.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return BF_ERR_CUDA;
        }
        int *ctrl = reinterpret_cast<int *>(scratch);
        const TcImg *imgs = reinterpret_cast<const TcImg *>(reinterpret_cast<char *>(scratch) + kCtrlWords * sizeof(int));
        if (d_sel == 6 && (rc = tc_ranges(imgs, keys, m, s)) != BF_OK) return rc;
        rc = tc_launch(imgs, m, total, ctrl, status, lay, variant, s);
        if (rc != BF_OK) return rc;
    }
    return BF_OK;
}

// ---------------------------------------------------------------------------------
// Allocation-free entry point
// ---------------------------------------------------------------------------------

// Scratch of bf_filter_batch_noalloc: control words (tile counter, status)
// followed by the image table and the six-channel range keys (12 words per
// image) for at most BF_NOALLOC_MAX_ITEMS images.  Every
// GPU that loads the library holds these 40.25 KB until the process exits.
constexpr size_t kNoAllocBytes =
    (size_t)kCtrlWords * sizeof(int) + (size_t)BF_NOALLOC_MAX_ITEMS * (sizeof(TcImg) + 12 * sizeof(uint32_t));
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
void *noalloc_scratch(int dev) {
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_noalloc_ptr[dev] = ptr;
    }
    return g_noalloc_ptr[dev];
}
}  // namespace

// Status word of the allocation-free entry point on the current device, or
// BF_OK if it was never used there; cleared when non-zero.
int noalloc_take_status() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BF_OK;
    void *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        p = g_noalloc_ptr[dev];
    }
    if (!p) return BF_OK;
    int v = 0;
    int *st = reinterpret_cast<int *>(p) + 1;
    if (cudaMemcpy(&v, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BF_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        cudaMemcpy(st, &zero, sizeof(int), cudaMemcpyHostToDevice);
    }
    return v;
}

}  // namespace bf

extern "C" int bf_filter_batch_noalloc(const bf_item *items, int n, int variant, void *stream) {
    using namespace bf;
    if (n < 0 || (n > 0 && !items)) return BF_ERR_ARG;
    if (variant != BF_FP16TC && variant != BF_BF16TC) return BF_ERR_ARG;
    if (n > BF_NOALLOC_MAX_ITEMS) return BF_ERR_BUDGET;
    cudaStream_t s = (cudaStream_t)stream;
    // The uploads below copy from this call's stack; a captured graph would
    // replay them after the frame is gone, so the call refuses capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return BF_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return BF_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const int rc = check_image_args(items[i].plan, items[i].in, items[i].out, items[i].H, items[i].W,
                                        items[i].pitch);
        if (rc != BF_OK) return rc;
    }
    TcImg tab[BF_NOALLOC_MAX_ITEMS];  // host staging on the stack: no heap allocation either
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BF_ERR_CUDA;
    char *scr = reinterpret_cast<char *>(noalloc_scratch(dev));
    if (!scr) return BF_ERR_CUDA;
    int *ctrl = reinterpret_cast<int *>(scr);
    TcImg *imgs = reinterpret_cast<TcImg *>(scr + kCtrlWords * sizeof(int));
    for (const int d_sel : {3, 6}) {  // as bf_filter_batch: one launch per channel count, in stream order
        int m = 0, total = 0;
        TcLayout lay{};
        int rc = tc_prepare(items, n, variant, d_sel, tab, &m, &total, &lay);
        if (rc != BF_OK) return rc;
        if (m == 0) continue;
        uint32_t *keys = reinterpret_cast<uint32_t *>(imgs + m);
        for (int i = 0; i < m; ++i) tab[i].mm = d_sel == 6 ? keys + 6 * i : nullptr;
        const int zero = 0;  // the tile counter must start at zero; the status word is left as is
        if (cudaMemcpyAsync(ctrl, &zero, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(imgs, tab, (size_t)m * sizeof(TcImg), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return BF_ERR_CUDA;
        }
        if (d_sel == 6 && (rc = tc_ranges(imgs, keys, m, s)) != BF_OK) return rc;
        rc = tc_launch(imgs, m, total, ctrl, ctrl + 1, lay, variant, s);
        if (rc != BF_OK) return rc;
    }
    return BF_OK;
}

namespace bf {

int launch_tc(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, int variant,
              cudaStream_t s) {
    bf_item it{const_cast<bf_plan_s *>(&p), in, out, H, W, pitch};
    void *scratch = stream_scratch(s, tc_scratch_bytes(1));
    int dev = 0;
    cudaGetDevice(&dev);
    int *st = status_word(dev);
    if (!scratch || !st) return BF_ERR_NOMEM;
    return tc_launch_batch(&it, 1, variant, scratch, st, s);
}

}  // namespace bf
