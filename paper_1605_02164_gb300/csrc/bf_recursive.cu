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
//   rec_cols  a block owns 16 columns; one thread per (column, channel) runs
//             the anticausal sections bottom to top into V, then the causal
//             ones top to bottom; each row's 2(d+1) blurred values meet in
//             shared memory and are combined with the centre cos/sin into the
//             P / Z accumulators (Eqs. numerator, denom, real parts).
//             Loads run 8 rows ahead of the recursion.
//   a final kernel divides P by Z.
// Scratch (library-owned, per stream): X and V (2(d+1) planes each) and P/Z
// (d + 1 planes), FP32, rows padded to 32.
#include <cuda_runtime.h>

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

constexpr int kRowT = 256;  // rec_rows: 32 rows x 8 channel groups
constexpr int kColT = 128;  // rec_cols: 16 columns x 8 channel groups
constexpr int kCols = 16;
constexpr int kAhead = 8;   // rows loaded ahead of the column recursion

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
                                                  int k, float *__restrict__ X, int Wp, Sections S) {
    constexpr int C2 = 2 * (D + 1);
    constexpr int CPT = (C2 + 7) / 8;  // channels per thread
    extern __shared__ float cb[];      // [C2][32][33]
    const int tid = threadIdx.x, y0 = blockIdx.x * 32;
    const size_t plane = (size_t)H * pitch, xplane = (size_t)H * Wp;
    float nh[D], nl[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        nh[c] = __ldg(nu_hi + k * D + c);
        nl[c] = __ldg(nu_lo + k * D + c);
    }
    auto build = [&](int cx) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = tid + kRowT * j, row = p >> 5, col = p & 31;
            const int gy = y0 + row, gx = cx + col;
            float fv[D], cs = 0.f, sn = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) fv[c] = 0.f;
            if (gy < H && gx < W) {
#pragma unroll
                for (int c = 0; c < D; ++c) fv[c] = __ldg(in + c * plane + (size_t)gy * pitch + gx);
                centre_cs<D>(fv, nh, nl, cs, sn);
            }
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
    for (int cx = 0; cx < W; cx += 32) {
        build(cx);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int ch = g + 8 * u;
            if (ch < C2) {
                float *line = cb + ch * 1056 + row * 33;
                for (int col = 0; col < 32; ++col) {
                    const float x = line[col];
                    const float y0v = fmaf(S.q0[0], x, fmaf(S.q1[0], xs[u], fmaf(-S.p1[0], a1[u], -S.p2[0] * a2[u])));
                    const float y1v = fmaf(S.q0[1], x, fmaf(S.q1[1], xs[u], fmaf(-S.p1[1], b1[u], -S.p2[1] * b2[u])));
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
    for (int cx = ((W - 1) / 32) * 32; cx >= 0; cx -= 32) {
        build(cx);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int ch = g + 8 * u;
            if (ch < C2) {
                float *line = cb + ch * 1056 + row * 33;
                for (int col = 31; col >= 0; --col) {
                    const float x = line[col];
                    const float v0 = fmaf(S.e1[0], x1[u], fmaf(S.e2[0], x2[u], fmaf(-S.p1[0], a1[u], -S.p2[0] * a2[u])));
                    const float v1 = fmaf(S.e1[1], x1[u], fmaf(S.e2[1], x2[u], fmaf(-S.p1[1], b1[u], -S.p2[1] * b2[u])));
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
        for (int ch = 0; ch < C2; ++ch)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = tid + kRowT * j, r = p >> 5, col = p & 31;
                if (y0 + r < H && cx + col < W) X[ch * xplane + (size_t)(y0 + r) * Wp + cx + col] += cb[ch * 1056 + r * 33 + col];
            }
        __syncthreads();
    }
}

template <int D>
__global__ void __launch_bounds__(kColT) rec_cols(const float *__restrict__ in, int pitch, int H, int W,
                                                  const float *__restrict__ nu_hi, const float *__restrict__ nu_lo,
                                                  int k, const float *__restrict__ X, float *__restrict__ V,
                                                  float *__restrict__ PZ, int Wp, Sections S) {
    constexpr int C2 = 2 * (D + 1);
    constexpr int CPT = (C2 + 7) / 8;
    constexpr int NPZ = (kCols * (D + 1) + kColT - 1) / kColT;  // P/Z values per thread per row
    __shared__ float sB[C2][kCols];
    __shared__ float2 sCS[kCols];
    const int tid = threadIdx.x, col = tid & (kCols - 1), g = tid >> 4;
    const int x = blockIdx.x * kCols + col;
    const bool xin = x < W;
    const size_t plane = (size_t)H * pitch, xplane = (size_t)H * Wp;
    float nh[D], nl[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        nh[c] = __ldg(nu_hi + k * D + c);
        nl[c] = __ldg(nu_lo + k * D + c);
    }

    // anticausal, bottom to top, into V
    float x1[CPT], x2[CPT], a1[CPT], a2[CPT], b1[CPT], b2[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) x1[u] = x2[u] = a1[u] = a2[u] = b1[u] = b2[u] = 0.f;
    for (int yb = H - 1; yb >= 0; yb -= kAhead) {
        float xv[CPT][kAhead];
#pragma unroll
        for (int u = 0; u < CPT; ++u)
#pragma unroll
            for (int a = 0; a < kAhead; ++a) {
                const int ch = g + 8 * u, y = yb - a;
                xv[u][a] = (ch < C2 && xin && y >= 0) ? X[ch * xplane + (size_t)y * Wp + x] : 0.f;
            }
#pragma unroll
        for (int a = 0; a < kAhead; ++a) {
            const int y = yb - a;
            if (y < 0) break;
#pragma unroll
            for (int u = 0; u < CPT; ++u) {
                const int ch = g + 8 * u;
                const float v0 = fmaf(S.e1[0], x1[u], fmaf(S.e2[0], x2[u], fmaf(-S.p1[0], a1[u], -S.p2[0] * a2[u])));
                const float v1 = fmaf(S.e1[1], x1[u], fmaf(S.e2[1], x2[u], fmaf(-S.p1[1], b1[u], -S.p2[1] * b2[u])));
                x2[u] = x1[u];
                x1[u] = xv[u][a];
                a2[u] = a1[u];
                a1[u] = v0;
                b2[u] = b1[u];
                b1[u] = v1;
                if (ch < C2 && xin) V[ch * xplane + (size_t)y * Wp + x] = v0 + v1;
            }
        }
    }
    __syncthreads();  // V of this block's columns is complete (each thread reads only its own values back)

    // causal, top to bottom, combined row by row into P / Z
    float xp[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) xp[u] = a1[u] = a2[u] = b1[u] = b2[u] = 0.f;
    for (int yb = 0; yb < H; yb += kAhead) {
        float xv[CPT][kAhead], vv[CPT][kAhead];
#pragma unroll
        for (int u = 0; u < CPT; ++u)
#pragma unroll
            for (int a = 0; a < kAhead; ++a) {
                const int ch = g + 8 * u, y = yb + a;
                const bool ok = ch < C2 && xin && y < H;
                xv[u][a] = ok ? X[ch * xplane + (size_t)y * Wp + x] : 0.f;
                vv[u][a] = ok ? V[ch * xplane + (size_t)y * Wp + x] : 0.f;
            }
        // centre values (group 0) and the P / Z accumulators of these rows
        float fc[kAhead][D];
        if (g == 0) {
#pragma unroll
            for (int a = 0; a < kAhead; ++a)
#pragma unroll
                for (int c = 0; c < D; ++c)
                    fc[a][c] = (xin && yb + a < H) ? __ldg(in + c * plane + (size_t)(yb + a) * pitch + x) : 0.f;
        }
        float acc[NPZ][kAhead];
#pragma unroll
        for (int i = 0; i < NPZ; ++i) {
            const int t = tid + kColT * i, cc = t >> 4, xx = blockIdx.x * kCols + (t & (kCols - 1));
#pragma unroll
            for (int a = 0; a < kAhead; ++a)
                acc[i][a] = (cc <= D && xx < W && yb + a < H) ? PZ[cc * xplane + (size_t)(yb + a) * Wp + xx] : 0.f;
        }
#pragma unroll
        for (int a = 0; a < kAhead; ++a) {
            const int y = yb + a;
            if (y >= H) break;
#pragma unroll
            for (int u = 0; u < CPT; ++u) {
                const int ch = g + 8 * u;
                const float xn = xv[u][a];
                const float y0v = fmaf(S.q0[0], xn, fmaf(S.q1[0], xp[u], fmaf(-S.p1[0], a1[u], -S.p2[0] * a2[u])));
                const float y1v = fmaf(S.q0[1], xn, fmaf(S.q1[1], xp[u], fmaf(-S.p1[1], b1[u], -S.p2[1] * b2[u])));
                xp[u] = xn;
                a2[u] = a1[u];
                a1[u] = y0v;
                b2[u] = b1[u];
                b1[u] = y1v;
                if (ch < C2) sB[ch][col] = y0v + y1v + vv[u][a];
            }
            if (g == 0) {
                float c_, s_;
                centre_cs<D>(fc[a], nh, nl, c_, s_);
                sCS[col] = make_float2(c_, s_);
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < NPZ; ++i) {
                const int t = tid + kColT * i, cc = t >> 4, cl = t & (kCols - 1);
                if (cc <= D) {
                    const float2 cs = sCS[cl];
                    acc[i][a] = fmaf(cs.x, sB[cc][cl], fmaf(cs.y, sB[D + 1 + cc][cl], acc[i][a]));
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < NPZ; ++i) {
            const int t = tid + kColT * i, cc = t >> 4, xx = blockIdx.x * kCols + (t & (kCols - 1));
#pragma unroll
            for (int a = 0; a < kAhead; ++a)
                if (cc <= D && xx < W && yb + a < H) PZ[cc * xplane + (size_t)(yb + a) * Wp + xx] = acc[i][a];
        }
    }
}

template <int D>
__global__ void rec_divide(const float *__restrict__ PZ, int Wp, float *__restrict__ out, int pitch, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const size_t xplane = (size_t)H * Wp, plane = (size_t)H * pitch;
    const float z = PZ[D * xplane + (size_t)y * Wp + x];
#pragma unroll
    for (int c = 0; c < D; ++c) out[c * plane + (size_t)y * pitch + x] = PZ[c * xplane + (size_t)y * Wp + x] / z;
}

template <int D>
int launch_d(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, cudaStream_t s) {
    constexpr int C2 = 2 * (D + 1);
    const int Wp = (W + 31) / 32 * 32;
    const size_t xplane = (size_t)H * Wp;
    const size_t bytes = (2 * C2 + (D + 1)) * xplane * sizeof(float);
    float *X = (float *)bf::stream_scratch(s, bytes);
    if (!X) return BF_ERR_NOMEM;
    float *V = X + C2 * xplane, *PZ = V + C2 * xplane;
    int rc = bf::cuda_err(cudaMemsetAsync(PZ, 0, (D + 1) * xplane * sizeof(float), s));
    if (rc != BF_OK) return rc;
    const Sections S = make_sections(p.sigma_s);
    const int smem = C2 * 32 * 33 * (int)sizeof(float);
    if (smem > 48 * 1024) {
        rc = bf::cuda_err(cudaFuncSetAttribute(rec_rows<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        if (rc != BF_OK) return rc;
    }
    const unsigned row_blocks = (unsigned)((H + 31) / 32), col_blocks = (unsigned)((W + kCols - 1) / kCols);
    for (int k = 0; k < p.K; ++k) {
        rec_rows<D><<<row_blocks, kRowT, smem, s>>>(in, pitch, H, W, p.nu_hi, p.nu_lo, k, X, Wp, S);
        rec_cols<D><<<col_blocks, kColT, 0, s>>>(in, pitch, H, W, p.nu_hi, p.nu_lo, k, X, V, PZ, Wp, S);
    }
    rec_divide<D><<<dim3((unsigned)((W + 127) / 128), (unsigned)H), 128, 0, s>>>(PZ, Wp, out, pitch, H, W);
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
