// Algorithm 1 with Deriche's recursive Gaussian in the convolution step: the
// O(1)-in-sigma_s variant the paper names for that step (Section 3, citing
// Deriche 1993).  FP32 throughout (variant BF_FP32_RECURSIVE).
//
// The filter.  Deriche fits the unnormalised Gaussian exp(-x^2 / 2 sigma^2),
// x >= 0, by two damped sinusoids in x / sigma with his published constants
// (a0 1.680, a1 3.735, b0 1.783, w0 0.6318, c0 -0.6803, c1 -0.2598, b1 1.723,
// w1 1.997) and filters with h(|n|) = causal part (n >= 0) + anticausal part
// (n <= -1).  Here each part is run as two second-order sections in parallel,
// one per damped sinusoid (the partial-fraction form of the 4th-order
// recursion: same filter, far better conditioned in FP32):
//   causal      y_i(n) = q_i0 x(n) + q_i1 x(n-1) - p_i1 y_i(n-1) - p_i2 y_i(n-2)
//   anticausal  v_i(n) = e_i1 x(n+1) + e_i2 x(n+2) - p_i1 v_i(n+1) - p_i2 v_i(n+2)
// (each evaluated as the part that does not depend on the previous output,
// then one FMA with it: one FMA per step on the recursion's critical path)
// with p_i1 = -2 e^{-beta_i} cos om_i, p_i2 = e^{-2 beta_i}, q_i0 = a,
// q_i1 = (c sin om_i - a cos om_i) e^{-beta_i}, e_i1 = q_i1 - q_i0 p_i1,
// e_i2 = -q_i0 p_i2 (the z-transform of e^{-beta n}(a cos om n + c sin om n)
// and of its tail n >= 1).  Zero state at both ends of a line: the image is
// zero outside, the truncation reading of the windowed filter.  The support is
// the whole image, so this is a different filter from the 3-sigma window.
//
// Work per term (whole image, two kernels):
//   rec_rows  a block owns 32 rows and walks them in 32-column chunks: builds
//             the 2(d+1) modulated channels of the chunk in shared memory
//             (phase as in the FP32 kernel: product residual + sincospif), one
//             thread per (row, channel) runs the causal sections left to right
//             and writes X; then right to left the anticausal sections, adding
//             into X.  Coalesced 128-byte row segments in and out.
//   rec_cols  one thread per column carries all 2(d+1) channels: the
//             anticausal sections bottom to top into V, then the causal ones
//             top to bottom, each row's blurred values combined at once with
//             the centre cos/sin into the P / Z accumulators (Eqs. numerator,
//             denom, real parts).  No barriers; loads run 2-4 rows ahead.
//   32 or more terms run per launch (grid.y), each with its own X, V and P / Z
//   slot, so more independent recursions are in flight and the sum over
//   terms has a fixed order; a final kernel adds the slots and divides.
// Scratch (library-owned, per stream, at most 24 GB): per term slot X and V
// (2(d+1) planes each) and P/Z (d + 1 planes), FP32, rows padded to 32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "bf.h"
#include "bf_internal.cuh"

namespace {

struct Sections {  // two parallel second-order sections (causal and anticausal parts)
    float q0[2], q1[2], e1[2], e2[2], p1[2], p2[2];
};

Sections make_sections(double sigma) {
    const double fit[2][4] = {{1.680, 3.735, 1.783, 0.6318},     // a, c, b, w of the first sinusoid
                              {-0.6803, -0.2598, 1.723, 1.997}};  // and of the second
    Sections S{};
    for (int i = 0; i < 2; ++i) {
        const double a = fit[i][0], c = fit[i][1], beta = fit[i][2] / sigma, om = fit[i][3] / sigma;
        const double p1 = -2.0 * std::exp(-beta) * std::cos(om), p2 = std::exp(-2.0 * beta);
        const double q0 = a, q1 = (c * std::sin(om) - a * std::cos(om)) * std::exp(-beta);
        S.q0[i] = (float)q0;
        S.q1[i] = (float)q1;
        S.e1[i] = (float)(q1 - q0 * p1);
        S.e2[i] = (float)(-q0 * p2);
        S.p1[i] = (float)p1;
        S.p2[i] = (float)p2;
    }
    return S;
}

constexpr int kRowT = 256;       // rec_rows: 32 rows x 8 channel groups
constexpr int kColT = 128;       // rec_cols: one column per thread
constexpr int kTermBatch = 32;   // terms per launch (grid.y), at least
constexpr int kColThreadsTarget = 152 * 4 * kColT;  // column threads wanted per launch
constexpr size_t kScratchCap = (size_t)24 << 30;  // bound on the per-stream scratch of this variant

// Phase of one pixel (turns), kept as in the FP32 kernel: FP32 product with its
// exact residual and explicit reduction to [-1/2, 1/2], then sincospif.
template <int D>
__device__ __forceinline__ void centre_cs(const float *fv, const float *nh, const float *nl, float &c, float &s) {
    float tf = 0.f, te = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float p = __fmul_rn(nh[k], fv[k]);
        const float e = fmaf(nh[k], fv[k], -p);
        tf = __fadd_rn(tf, __fsub_rn(p, rintf(p)));
        tf = __fsub_rn(tf, rintf(tf));
        te = fmaf(nl[k], fv[k], __fadd_rn(te, e));
    }
    sincospif(2.f * __fadd_rn(tf, te), &s, &c);
}

// Channel order: cos th f_0..f_{d-1}, cos th, sin th f_0..f_{d-1}, sin th.
template <int D>
__global__ void __launch_bounds__(kRowT) rec_rows(const float *__restrict__ in, int pitch, int H, int W,
                                                  const float *__restrict__ nu_hi, const float *__restrict__ nu_lo,
                                                  int k0, float *__restrict__ X, int Wp, size_t term_stride,
                                                  Sections S) {
    constexpr int C2 = 2 * (D + 1);
    constexpr int CPT = (C2 + 7) / 8;  // channels per thread
    extern __shared__ float cb[];      // [C2][32][33]
    const int tid = threadIdx.x, y0 = blockIdx.x * 32, k = k0 + blockIdx.y;
    X += blockIdx.y * term_stride;
    const size_t plane = (size_t)H * pitch, xplane = (size_t)H * Wp;
    float nh[D], nl[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        nh[c] = __ldg(nu_hi + k * D + c);
        nl[c] = __ldg(nu_lo + k * D + c);
    }
    // f of this thread's 4 pixels of a chunk, loaded one chunk ahead of build
    float fpf[4][D];
    auto load_f = [&](int cx) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = tid + kRowT * j, gy = y0 + (p >> 5), gx = cx + (p & 31);
            const bool ok = gy < H && gx < W;
#pragma unroll
            for (int c = 0; c < D; ++c) fpf[j][c] = ok ? __ldg(in + c * plane + (size_t)gy * pitch + gx) : 0.f;
        }
    };
    auto build = [&](int cx) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = tid + kRowT * j, row = p >> 5, col = p & 31;
            const float *fv = fpf[j];
            float cs = 0.f, sn = 0.f;
            if (y0 + row < H && cx + col < W) centre_cs<D>(fv, nh, nl, cs, sn);
            float *d = cb + row * 33 + col;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                d[c * 1056] = cs * fv[c];
                d[(D + 1 + c) * 1056] = sn * fv[c];
            }
            d[D * 1056] = cs;
            d[(2 * D + 1) * 1056] = sn;
        }
    };
    const int row = tid & 31, g = tid >> 5;
    // causal: x(n-1), y_0(n-1), y_0(n-2), y_1(n-1), y_1(n-2) per channel
    float xs[CPT], a1[CPT], a2[CPT], b1[CPT], b2[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) xs[u] = a1[u] = a2[u] = b1[u] = b2[u] = 0.f;
    load_f(0);
    for (int cx = 0; cx < W; cx += 32) {
        build(cx);
        if (cx + 32 < W) load_f(cx + 32);  // in flight during the recursion and the stores
        __syncthreads();
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int ch = g + 8 * u;
            if (ch < C2) {
                float *line = cb + ch * 1056 + row * 33;
#pragma unroll
                for (int col = 0; col < 32; ++col) {
                    const float x = line[col];
                    const float y0v = fmaf(-S.p1[0], a1[u], fmaf(S.q0[0], x, fmaf(S.q1[0], xs[u], -S.p2[0] * a2[u])));
                    const float y1v = fmaf(-S.p1[1], b1[u], fmaf(S.q0[1], x, fmaf(S.q1[1], xs[u], -S.p2[1] * b2[u])));
                    xs[u] = x;
                    a2[u] = a1[u];
                    a1[u] = y0v;
                    b2[u] = b1[u];
                    b1[u] = y1v;
                    line[col] = y0v + y1v;
                }
            }
        }
        __syncthreads();
        for (int ch = 0; ch < C2; ++ch)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = tid + kRowT * j, r = p >> 5, col = p & 31;
                if (y0 + r < H && cx + col < W) X[ch * xplane + (size_t)(y0 + r) * Wp + cx + col] = cb[ch * 1056 + r * 33 + col];
            }
        __syncthreads();
    }
    // anticausal: x(n+1), x(n+2), v_0(n+1), v_0(n+2), v_1(n+1), v_1(n+2)
    float x1[CPT], x2[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) x1[u] = x2[u] = a1[u] = a2[u] = b1[u] = b2[u] = 0.f;
    load_f(((W - 1) / 32) * 32);
    for (int cx = ((W - 1) / 32) * 32; cx >= 0; cx -= 32) {
        build(cx);
        // the causal results this thread adds to, loaded before the recursion
        float xr[C2][4];
#pragma unroll
        for (int ch = 0; ch < C2; ++ch)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = tid + kRowT * j, r = p >> 5, col = p & 31;
                xr[ch][j] = (y0 + r < H && cx + col < W) ? X[ch * xplane + (size_t)(y0 + r) * Wp + cx + col] : 0.f;
            }
        if (cx >= 32) load_f(cx - 32);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int ch = g + 8 * u;
            if (ch < C2) {
                float *line = cb + ch * 1056 + row * 33;
#pragma unroll
                for (int col = 31; col >= 0; --col) {
                    const float x = line[col];
                    const float v0 = fmaf(-S.p1[0], a1[u], fmaf(S.e1[0], x1[u], fmaf(S.e2[0], x2[u], -S.p2[0] * a2[u])));
                    const float v1 = fmaf(-S.p1[1], b1[u], fmaf(S.e1[1], x1[u], fmaf(S.e2[1], x2[u], -S.p2[1] * b2[u])));
                    x2[u] = x1[u];
                    x1[u] = x;
                    a2[u] = a1[u];
                    a1[u] = v0;
                    b2[u] = b1[u];
                    b1[u] = v1;
                    line[col] = v0 + v1;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int ch = 0; ch < C2; ++ch)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = tid + kRowT * j, r = p >> 5, col = p & 31;
                if (y0 + r < H && cx + col < W)
                    X[ch * xplane + (size_t)(y0 + r) * Wp + cx + col] = xr[ch][j] + cb[ch * 1056 + r * 33 + col];
            }
        __syncthreads();
    }
}

template <int D>
__global__ void __launch_bounds__(kColT) rec_cols(const float *__restrict__ in, int pitch, int H, int W,
                                                  const float *__restrict__ nu_hi, const float *__restrict__ nu_lo,
                                                  int k0, const float *__restrict__ X, float *__restrict__ V,
                                                  float *__restrict__ PZ, int Wp, size_t term_stride, size_t pz_stride,
                                                  Sections S) {
    constexpr int C2 = 2 * (D + 1);
    constexpr int AA = C2 <= 8 ? 4 : 2;  // rows loaded ahead of the anticausal recursion
    constexpr int A = C2 <= 4 ? 4 : 2;   // and of the causal one (more live values)
    const int x = blockIdx.x * kColT + threadIdx.x;
    if (x >= W) return;  // no barriers in this kernel
    const int j = blockIdx.y, k = k0 + j;
    const float *Xj = X + j * term_stride;
    float *Vj = V + j * term_stride;
    float *PZj = PZ + j * pz_stride;
    const size_t plane = (size_t)H * pitch, xplane = (size_t)H * Wp;
    float nh[D], nl[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        nh[c] = __ldg(nu_hi + k * D + c);
        nl[c] = __ldg(nu_lo + k * D + c);
    }

    // anticausal, bottom to top, into V: x(n+1), x(n+2), v_0(n+1), v_0(n+2), v_1(n+1), v_1(n+2)
    float x1[C2], x2[C2], a1[C2], a2[C2], b1[C2], b2[C2];
#pragma unroll
    for (int c = 0; c < C2; ++c) x1[c] = x2[c] = a1[c] = a2[c] = b1[c] = b2[c] = 0.f;
    for (int yb = H - 1; yb >= 0; yb -= AA) {
        float xv[AA][C2];
#pragma unroll
        for (int a = 0; a < AA; ++a)
#pragma unroll
            for (int c = 0; c < C2; ++c) xv[a][c] = (yb - a >= 0) ? Xj[c * xplane + (size_t)(yb - a) * Wp + x] : 0.f;
#pragma unroll
        for (int a = 0; a < AA; ++a) {
            const int y = yb - a;
            if (y < 0) break;
#pragma unroll
            for (int c = 0; c < C2; ++c) {
                const float v0 = fmaf(-S.p1[0], a1[c], fmaf(S.e1[0], x1[c], fmaf(S.e2[0], x2[c], -S.p2[0] * a2[c])));
                const float v1 = fmaf(-S.p1[1], b1[c], fmaf(S.e1[1], x1[c], fmaf(S.e2[1], x2[c], -S.p2[1] * b2[c])));
                x2[c] = x1[c];
                x1[c] = xv[a][c];
                a2[c] = a1[c];
                a1[c] = v0;
                b2[c] = b1[c];
                b1[c] = v1;
                Vj[c * xplane + (size_t)y * Wp + x] = v0 + v1;
            }
        }
    }

    // causal, top to bottom, combined with the centre cos/sin into P / Z
#pragma unroll
    for (int c = 0; c < C2; ++c) x1[c] = a1[c] = a2[c] = b1[c] = b2[c] = 0.f;  // x1 = x(n-1) here
    for (int yb = 0; yb < H; yb += A) {
        float xv[A][C2], vv[A][C2], fv[A][D], pz[A][D + 1];
#pragma unroll
        for (int a = 0; a < A; ++a) {
            const bool ok = yb + a < H;
            const size_t o = (size_t)(yb + a) * Wp + x;
#pragma unroll
            for (int c = 0; c < C2; ++c) {
                xv[a][c] = ok ? Xj[c * xplane + o] : 0.f;
                vv[a][c] = ok ? Vj[c * xplane + o] : 0.f;
            }
#pragma unroll
            for (int c = 0; c <= D; ++c) pz[a][c] = ok ? PZj[c * xplane + o] : 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) fv[a][c] = ok ? __ldg(in + c * plane + (size_t)(yb + a) * pitch + x) : 0.f;
        }
#pragma unroll
        for (int a = 0; a < A; ++a) {
            if (yb + a >= H) break;
            float B[C2];
#pragma unroll
            for (int c = 0; c < C2; ++c) {
                const float xn = xv[a][c];
                const float y0v = fmaf(-S.p1[0], a1[c], fmaf(S.q0[0], xn, fmaf(S.q1[0], x1[c], -S.p2[0] * a2[c])));
                const float y1v = fmaf(-S.p1[1], b1[c], fmaf(S.q0[1], xn, fmaf(S.q1[1], x1[c], -S.p2[1] * b2[c])));
                x1[c] = xn;
                a2[c] = a1[c];
                a1[c] = y0v;
                b2[c] = b1[c];
                b1[c] = y1v;
                B[c] = y0v + y1v + vv[a][c];
            }
            float cs, sn;
            centre_cs<D>(fv[a], nh, nl, cs, sn);
#pragma unroll
            for (int c = 0; c <= D; ++c) pz[a][c] = fmaf(cs, B[c], fmaf(sn, B[D + 1 + c], pz[a][c]));
        }
#pragma unroll
        for (int a = 0; a < A; ++a)
            if (yb + a < H) {
                const size_t o = (size_t)(yb + a) * Wp + x;
#pragma unroll
                for (int c = 0; c <= D; ++c) PZj[c * xplane + o] = pz[a][c];
            }
    }
}

// out_c = sum_j P_j,c / sum_j Z_j over the term slots.
template <int D>
__global__ void rec_divide(const float *__restrict__ PZ, int Wp, size_t pz_stride, int slots, float *__restrict__ out,
                           int pitch, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const size_t xplane = (size_t)H * Wp, plane = (size_t)H * pitch, o = (size_t)y * Wp + x;
    float acc[D + 1];
#pragma unroll
    for (int c = 0; c <= D; ++c) acc[c] = 0.f;
    for (int j = 0; j < slots; ++j)
#pragma unroll
        for (int c = 0; c <= D; ++c) acc[c] += PZ[j * pz_stride + c * xplane + o];
#pragma unroll
    for (int c = 0; c < D; ++c) out[c * plane + (size_t)y * pitch + x] = acc[c] / acc[D];
}

template <int D>
int launch_d(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, cudaStream_t s) {
    constexpr int C2 = 2 * (D + 1);
    const int Wp = (W + 31) / 32 * 32;
    const size_t xplane = (size_t)H * Wp;
    const size_t term_stride = C2 * xplane, pz_stride = (D + 1) * xplane;
    // Terms run kTermBatch at a time (grid.y), each with its own X, V and P/Z
    // slot: more independent recursions in flight, and a fixed summation order.
    const size_t per_term = (2 * term_stride + pz_stride) * sizeof(float);
    // A narrow image gets more terms per launch, so that its column kernel
    // (one thread per column and term) still has ~4 blocks per SM.
    int tb = std::max(kTermBatch, (kColThreadsTarget + W - 1) / W);
    if (tb > p.K) tb = p.K;
    while (tb > 1 && (size_t)tb * per_term > kScratchCap) --tb;
    float *X = (float *)bf::stream_scratch(s, (size_t)tb * per_term);
    if (!X) return BF_ERR_NOMEM;
    float *V = X + (size_t)tb * term_stride, *PZ = V + (size_t)tb * term_stride;
    int rc = bf::cuda_err(cudaMemsetAsync(PZ, 0, (size_t)tb * pz_stride * sizeof(float), s));
    if (rc != BF_OK) return rc;
    const Sections S = make_sections(p.sigma_s);
    const int smem = C2 * 32 * 33 * (int)sizeof(float);
    if (smem > 48 * 1024) {
        rc = bf::cuda_err(cudaFuncSetAttribute(rec_rows<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        if (rc != BF_OK) return rc;
    }
    const unsigned row_blocks = (unsigned)((H + 31) / 32), col_blocks = (unsigned)((W + kColT - 1) / kColT);
    for (int k0 = 0; k0 < p.K; k0 += tb) {
        const unsigned nb = (unsigned)(p.K - k0 < tb ? p.K - k0 : tb);
        rec_rows<D><<<dim3(row_blocks, nb), kRowT, smem, s>>>(in, pitch, H, W, p.nu_hi, p.nu_lo, k0, X, Wp,
                                                              term_stride, S);
        rec_cols<D><<<dim3(col_blocks, nb), kColT, 0, s>>>(in, pitch, H, W, p.nu_hi, p.nu_lo, k0, X, V, PZ, Wp,
                                                           term_stride, pz_stride, S);
    }
    rec_divide<D><<<dim3((unsigned)((W + 127) / 128), (unsigned)H), 128, 0, s>>>(PZ, Wp, pz_stride, tb, out, pitch,
                                                                                 H, W);
    return bf::cuda_err(cudaGetLastError());
}

}  // namespace

namespace bf {

int launch_recursive(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, cudaStream_t s) {
    if (H > 65535) return BF_ERR_UNSUPPORTED;  // grid.y of the final division
    switch (p.d) {
        case 1: return launch_d<1>(p, in, out, H, W, pitch, s);
        case 2: return launch_d<2>(p, in, out, H, W, pitch, s);
        case 3: return launch_d<3>(p, in, out, H, W, pitch, s);
        case 4: return launch_d<4>(p, in, out, H, W, pitch, s);
        case 5: return launch_d<5>(p, in, out, H, W, pitch, s);
        case 6: return launch_d<6>(p, in, out, H, W, pitch, s);
        case 7: return launch_d<7>(p, in, out, H, W, pitch, s);
        case 8: return launch_d<8>(p, in, out, H, W, pitch, s);
        default: return BF_ERR_D_RANGE;
    }
}

}  // namespace bf
