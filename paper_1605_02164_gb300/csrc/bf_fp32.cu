// Fused FP32 kernel for the Monte Carlo shiftable bilateral filter
// (Algorithm 1; Eqs. Ht, numerator, denom), every step on the CUDA cores.
//
// One CTA owns a tile of kBX x BY output pixels and keeps, across all K
// terms, its accumulators P_1..P_d, Z in shared memory.  For each term it
// streams the tile's input region (tile plus an r-pixel halo) down in chunks
// of kRC rows:
//   A  phase theta = 2 pi nu_t . f (FP32 with an exact product residual and
//      explicit range reduction), cos/sin once per pixel, and the 2(d+1)
//      modulated channels cos th f_c, cos th, sin th f_c, sin th  (zero
//      outside the image: neighbours outside Omega drop out of both sums);
//   B  horizontal Gaussian pass of the chunk into a ring of row results;
//   C  vertical pass over the ring for the output rows that became complete,
//      combined with the centre pixel's cos/sin:  P_c += cos th(i) Bc_c(i) +
//      sin th(i) Bs_c(i),  Z += cos th(i) Bc(i) + sin th(i) Bs(i).
// After the last term out_c = P_c / Z (the 1/K factors cancel).
// Both passes are register-blocked: a thread produces 8 consecutive outputs
// from a sliding 16-value register window, 8 taps per step (taps past 2r are
// zero).  HBM sees the input once per term through L2 and the output once.
// When the 2(d+1) channels of a chunk do not fit in shared memory (large d
// and r), each term runs in two passes (G = 2): the cos-group channels
// cos f_c, cos and then the sin-group channels sin f_c, sin, each pass adding
// its half of P and Z (cos/sin are recomputed in the second pass).
#include <cuda_runtime.h>
#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kThreads = 512;
constexpr int kRC = 16;  // region rows per chunk
constexpr int kBX = 32;  // output columns per tile

struct Geom {
    int r, BY, RX, U8, TP, RXP, RING, RING_CS, lag, NJ, HB_SLOT;
    size_t smem_floats;
};

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

template <int D, int G>
Geom make_geom(int r, int BY) {
    Geom g;
    constexpr int NCH = 2 * (D + 1) / G;  // channels held per pass
    g.r = r;
    g.BY = BY;
    g.RX = kBX + 2 * r;
    g.U8 = cdiv(2 * r + 1, 8);
    g.TP = 8 * g.U8;
    g.RXP = kBX + 8 * g.U8 + 4;  // covers every column the sliding window reads; %32 == 4 spreads banks
    g.lag = cdiv(2 * r, kRC);
    g.RING = kRC * (g.lag + 1);
    g.RING_CS = g.RING + kRC;
    g.NJ = cdiv(BY + 2 * r, kRC);
    g.HB_SLOT = NCH * kBX + 4;
    g.smem_floats = (size_t)g.TP + (size_t)NCH * kRC * g.RXP + (size_t)g.RING * g.HB_SLOT +
                    (size_t)g.RING_CS * kBX * 2 + (size_t)(D + 1) * BY * kBX;
    return g;
}

template <int D, int G>
__global__ void __launch_bounds__(kThreads, 1)
    mcsf_fp32_kernel(const float *__restrict__ in, float *__restrict__ out, int H, int W, int pitch,
                     const float *__restrict__ nu_hi, const float *__restrict__ nu_lo, int K,
                     const float *__restrict__ taps_g, Geom g) {
    constexpr int NCH = 2 * (D + 1) / G;  // channels held per pass
    extern __shared__ __align__(16) float smem[];
    float *taps = smem;                                   // [TP]
    float *CH = taps + g.TP;                              // [NCH][kRC][RXP]
    float *HB = CH + (size_t)NCH * kRC * g.RXP;           // [RING][HB_SLOT] (= [NCH][kBX] + pad)
    float2 *CS = reinterpret_cast<float2 *>(HB + (size_t)g.RING * g.HB_SLOT);  // [RING_CS][kBX]
    float *ACC = reinterpret_cast<float *>(CS + (size_t)g.RING_CS * kBX);      // [D+1][BY][kBX]

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int r = g.r, BY = g.BY;
    const int tx0 = blockIdx.x * kBX, ty0 = blockIdx.y * BY;
    const size_t plane = (size_t)H * pitch;

    for (int i = tid; i < g.TP; i += kThreads) taps[i] = taps_g[i];
    for (int i = tid; i < g.RING * g.HB_SLOT; i += kThreads) HB[i] = 0.f;
    for (int i = tid; i < (D + 1) * BY * kBX; i += kThreads) ACC[i] = 0.f;
    __syncthreads();

    for (int k = 0; k < K; ++k) {
        float nh[D], nl[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            nh[c] = __ldg(nu_hi + k * D + c);
            nl[c] = __ldg(nu_lo + k * D + c);
        }
      for (int gi = 0; gi < G; ++gi) {  // channel group of this pass (G = 1: both groups at once)
        for (int j = 0; j < g.NJ; ++j) {
            // ---------------- A: phases, cos/sin, modulated channels ----------
            const int ring0 = (j * kRC) % g.RING;
            const int cs0 = (j * kRC) % g.RING_CS;
            for (int row = warp; row < kRC; row += kThreads / 32) {
                const int ry = j * kRC + row;
                const int gy = ty0 - r + ry;
                const bool rowok = ry < BY + 2 * r && gy >= 0 && gy < H;
                for (int col = lane; col < g.RXP; col += 32) {
                    const int gx = tx0 - r + col;
                    float cth = 0.f, sth = 0.f, fv[D];
#pragma unroll
                    for (int c = 0; c < D; ++c) fv[c] = 0.f;
                    if (rowok && col < g.RX && gx >= 0 && gx < W) {
                        const float *px = in + (size_t)gy * pitch + gx;
#pragma unroll
                        for (int c = 0; c < D; ++c) fv[c] = __ldg(px + c * plane);
                        // t = nu . f mod 1, with the FP32 product residual kept
                        float tf = 0.f, te = 0.f;
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            const float p = __fmul_rn(nh[c], fv[c]);
                            const float e = fmaf(nh[c], fv[c], -p);        // exact: nh*f - p
                            tf = __fadd_rn(tf, __fsub_rn(p, rintf(p)));    // |.| <= 1
                            tf = __fsub_rn(tf, rintf(tf));                 // back to [-1/2, 1/2]
                            te = fmaf(nl[c], fv[c], __fadd_rn(te, e));
                        }
                        sincospif(2.f * __fadd_rn(tf, te), &sth, &cth);
                    }
                    float *dst = CH + row * g.RXP + col;
                    if (G == 1) {
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            dst[(size_t)c * kRC * g.RXP] = cth * fv[c];
                            dst[(size_t)(D + 1 + c) * kRC * g.RXP] = sth * fv[c];
                        }
                        dst[(size_t)D * kRC * g.RXP] = cth;
                        dst[(size_t)(2 * D + 1) * kRC * g.RXP] = sth;
                    } else {
                        const float trig = gi == 0 ? cth : sth;
#pragma unroll
                        for (int c = 0; c < D; ++c) dst[(size_t)c * kRC * g.RXP] = trig * fv[c];
                        dst[(size_t)D * kRC * g.RXP] = trig;
                    }
                    const int cx = col - r;
                    if (cx >= 0 && cx < kBX) CS[(cs0 + row) * kBX + cx] = make_float2(cth, sth);
                }
            }
            __syncthreads();
            // ---------------- B: horizontal pass into the ring ---------------
            for (int task = tid; task < kRC * NCH * (kBX / 8); task += kThreads) {
                const int xb = task & 3;
                const int row = (task >> 2) & (kRC - 1);
                const int ch = task >> 6;
                const float *src = CH + ((size_t)ch * kRC + row) * g.RXP + xb * 8;
                float acc[8], win[16];
#pragma unroll
                for (int m = 0; m < 8; ++m) acc[m] = 0.f;
                *reinterpret_cast<float4 *>(&win[0]) = *reinterpret_cast<const float4 *>(src);
                *reinterpret_cast<float4 *>(&win[4]) = *reinterpret_cast<const float4 *>(src + 4);
                for (int u0 = 0; u0 < g.TP; u0 += 8) {
                    *reinterpret_cast<float4 *>(&win[8]) = *reinterpret_cast<const float4 *>(src + u0 + 8);
                    *reinterpret_cast<float4 *>(&win[12]) = *reinterpret_cast<const float4 *>(src + u0 + 12);
                    const float4 ta = *reinterpret_cast<const float4 *>(taps + u0);
                    const float4 tb = *reinterpret_cast<const float4 *>(taps + u0 + 4);
                    const float tv[8] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z, tb.w};
#pragma unroll
                    for (int uu = 0; uu < 8; ++uu)
#pragma unroll
                        for (int m = 0; m < 8; ++m) acc[m] = fmaf(tv[uu], win[m + uu], acc[m]);
#pragma unroll
                    for (int m = 0; m < 8; ++m) win[m] = win[m + 8];
                }
                float *dst = HB + (size_t)(ring0 + row) * g.HB_SLOT + ch * kBX + xb * 8;
                *reinterpret_cast<float4 *>(dst) = make_float4(acc[0], acc[1], acc[2], acc[3]);
                *reinterpret_cast<float4 *>(dst + 4) = make_float4(acc[4], acc[5], acc[6], acc[7]);
            }
            __syncthreads();
            // ---------------- C: vertical pass + combine ----------------------
            const int oc = j - g.lag;
            if (oc >= 0 && oc * kRC < BY) {
                if (G == 1) {
                    for (int task = tid; task < kBX * (D + 1) * 2; task += kThreads) {
                        const int x = task & 31;
                        const int rb = (task >> 5) & 1;
                        const int p = task >> 6;
                        const int o0 = oc * kRC + rb * 8;
                        const float *hc = HB + p * kBX + x;            // cos-group channel p
                        const float *hs = HB + (D + 1 + p) * kBX + x;  // sin-group channel p
                        float vc[8], vs[8], wc[16], ws[16];
                        int blk = o0 % g.RING;
    #pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            vc[m] = 0.f;
                            vs[m] = 0.f;
                            wc[m] = hc[(size_t)(blk + m) * g.HB_SLOT];
                            ws[m] = hs[(size_t)(blk + m) * g.HB_SLOT];
                        }
                        for (int v0 = 0; v0 < g.TP; v0 += 8) {
                            blk += 8;
                            if (blk >= g.RING) blk -= g.RING;
    #pragma unroll
                            for (int m = 0; m < 8; ++m) {
                                wc[8 + m] = hc[(size_t)(blk + m) * g.HB_SLOT];
                                ws[8 + m] = hs[(size_t)(blk + m) * g.HB_SLOT];
                            }
                            const float4 ta = *reinterpret_cast<const float4 *>(taps + v0);
                            const float4 tb = *reinterpret_cast<const float4 *>(taps + v0 + 4);
                            const float tv[8] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z, tb.w};
    #pragma unroll
                            for (int vv = 0; vv < 8; ++vv)
    #pragma unroll
                                for (int m = 0; m < 8; ++m) {
                                    vc[m] = fmaf(tv[vv], wc[m + vv], vc[m]);
                                    vs[m] = fmaf(tv[vv], ws[m + vv], vs[m]);
                                }
    #pragma unroll
                            for (int m = 0; m < 8; ++m) {
                                wc[m] = wc[m + 8];
                                ws[m] = ws[m + 8];
                            }
                        }
                        int crow = (o0 + r) % g.RING_CS;
                        float *acc = ACC + ((size_t)p * BY + o0) * kBX + x;
    #pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            const float2 cs = CS[crow * kBX + x];
                            acc[m * kBX] += fmaf(cs.x, vc[m], cs.y * vs[m]);
                            if (++crow == g.RING_CS) crow = 0;
                        }
                    }
                } else {
                    // one channel group: V = blur of (trig f_p or trig), acc += trig(centre) V
                    for (int task = tid; task < kBX * (D + 1) * 2; task += kThreads) {
                        const int x = task & 31;
                        const int rb = (task >> 5) & 1;
                        const int p = task >> 6;
                        const int o0 = oc * kRC + rb * 8;
                        const float *hc = HB + p * kBX + x;
                        float vc[8], wc[16];
                        int blk = o0 % g.RING;
#pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            vc[m] = 0.f;
                            wc[m] = hc[(size_t)(blk + m) * g.HB_SLOT];
                        }
                        for (int v0 = 0; v0 < g.TP; v0 += 8) {
                            blk += 8;
                            if (blk >= g.RING) blk -= g.RING;
#pragma unroll
                            for (int m = 0; m < 8; ++m) wc[8 + m] = hc[(size_t)(blk + m) * g.HB_SLOT];
                            const float4 ta = *reinterpret_cast<const float4 *>(taps + v0);
                            const float4 tb = *reinterpret_cast<const float4 *>(taps + v0 + 4);
                            const float tv[8] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z, tb.w};
#pragma unroll
                            for (int vv = 0; vv < 8; ++vv)
#pragma unroll
                                for (int m = 0; m < 8; ++m) vc[m] = fmaf(tv[vv], wc[m + vv], vc[m]);
#pragma unroll
                            for (int m = 0; m < 8; ++m) wc[m] = wc[m + 8];
                        }
                        int crow = (o0 + r) % g.RING_CS;
                        float *acc = ACC + ((size_t)p * BY + o0) * kBX + x;
#pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            const float2 cs = CS[crow * kBX + x];
                            acc[m * kBX] += (gi == 0 ? cs.x : cs.y) * vc[m];
                            if (++crow == g.RING_CS) crow = 0;
                        }
                    }
                }
            }
            // no barrier here: the next chunk's A writes CH (read only by B)
            // and CS slots that C does not read (RING_CS has one spare chunk);
            // the barrier after that A orders this C before the next B.
        }
        __syncthreads();  // pass / term boundary: CS/HB slots are reused from row 0
      }
    }
    // ---------------- divide and store -----------------------------------------
    for (int idx = tid; idx < BY * kBX; idx += kThreads) {
        const int y = idx / kBX, x = idx % kBX;
        const int gy = ty0 + y, gx = tx0 + x;
        if (gy < H && gx < W) {
            const float z = ACC[((size_t)D * BY + y) * kBX + x];
#pragma unroll
            for (int c = 0; c < D; ++c)
                out[c * plane + (size_t)gy * pitch + gx] = ACC[((size_t)c * BY + y) * kBX + x] / z;
        }
    }
}

// Tallest tile (multiple of kRC, at most 128 rows) whose buffers fit; 0 if none.
template <int D, int G>
int fit_rows(int r, int H, int max_smem) {
    int BY = 128;
    while (BY >= kRC && make_geom<D, G>(r, BY).smem_floats * sizeof(float) > (size_t)max_smem) BY -= kRC;
    if (BY < kRC) return 0;
    const int by = kRC * cdiv(H, kRC);  // short image: no taller than needed
    return by < BY ? by : BY;
}

// Tile height for the SMs (one CTA per SM): among multiples of 16 rows up to BY,
// the one that minimises (waves of tiles) x (16-row chunks of phase and
// horizontal work + 16-row blocks of vertical work per tile), so that a small
// image spreads over all SMs.  A pixel's arithmetic does not depend on it.
int fit_waves(int r, int H, int W, int BY) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        return BY;
    }
    long long best = -1;
    int best_by = BY;
    for (int by = BY; by >= kRC; by -= kRC) {
        const long long tiles = (long long)cdiv(W, kBX) * cdiv(H, by);
        const long long cost = (tiles + nsm - 1) / nsm * (cdiv(by + 2 * r, kRC) + by / kRC);
        if (best < 0 || cost < best) {
            best = cost;
            best_by = by;
        }
    }
    return best_by;
}

template <int D, int G>
int launch_dg(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, int BY, cudaStream_t s,
              bool alone) {
    const int tuned = tune_rows(BF_FP32, D, p.r, H, W, alone ? BF_TUNE_ALONE : BF_TUNE_BATCH);
    if (tuned > 0)
        BY = tuned < BY ? tuned : BY;  // a measured height, within what fits
    else if (alone)
        BY = fit_waves(p.r, H, W, BY);
    const Geom g = make_geom<D, G>(p.r, BY);
    const size_t bytes = g.smem_floats * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(mcsf_fp32_kernel<D, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BF_ERR_CUDA;
    }
    dim3 grid(cdiv(W, kBX), cdiv(H, BY));
    mcsf_fp32_kernel<D, G><<<grid, kThreads, bytes, s>>>(in, out, H, W, pitch, p.nu_hi, p.nu_lo, p.K, p.taps, g);
    return cuda_err(cudaGetLastError());
}

// One pass per term when a tile of at least 32 rows fits, else two passes
// (channel groups), else BF_ERR_UNSUPPORTED.
template <int D>
int launch_d(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, cudaStream_t s, bool alone) {
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int by1 = fit_rows<D, 1>(p.r, H, max_smem);
    if (by1 >= 32 || (by1 > 0 && by1 >= kRC * cdiv(H, kRC))) return launch_dg<D, 1>(p, in, out, H, W, pitch, by1, s, alone);
    const int by2 = fit_rows<D, 2>(p.r, H, max_smem);
    if (by2 > 0) return launch_dg<D, 2>(p, in, out, H, W, pitch, by2, s, alone);
    if (by1 > 0) return launch_dg<D, 1>(p, in, out, H, W, pitch, by1, s, alone);
    return BF_ERR_UNSUPPORTED;
}

}  // namespace

int launch_fp32(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, cudaStream_t s, bool alone) {
    switch (p.d) {
        case 1: return launch_d<1>(p, in, out, H, W, pitch, s, alone);
        case 2: return launch_d<2>(p, in, out, H, W, pitch, s, alone);
        case 3: return launch_d<3>(p, in, out, H, W, pitch, s, alone);
        case 4: return launch_d<4>(p, in, out, H, W, pitch, s, alone);
        case 5: return launch_d<5>(p, in, out, H, W, pitch, s, alone);
        case 6: return launch_d<6>(p, in, out, H, W, pitch, s, alone);
        case 7: return launch_d<7>(p, in, out, H, W, pitch, s, alone);
        case 8: return launch_d<8>(p, in, out, H, W, pitch, s, alone);
        default: return BF_ERR_D_RANGE;
    }
}

}  // namespace bf
