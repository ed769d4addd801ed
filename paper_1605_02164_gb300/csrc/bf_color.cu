// sRGB (0..255) <-> CIE 1976 L*a*b* for filtering in Lab (Section 4, Fig. 4).
//
// The paper filters its House example in CIE-Lab and converts back, without
// naming the RGB space.  Here the RGB values are sRGB on the 0..255 scale:
// IEC 61966-2-1's piecewise transfer function and its D65 RGB -> XYZ matrix
// (printed there to four decimals), the white point is the XYZ of RGB white
// (the matrix row sums, so white maps to L* = 100, a* = b* = 0 exactly), and
// the CIE 1976 companding uses delta = 6/29.  Nothing is clipped, so values
// the filter leaves outside the gamut survive the round trip.
//
// Both directions are elementwise and bound by HBM: 12 bytes read and 12
// written per pixel.  One thread converts 4 consecutive pixels of a row with
// 16-byte loads and stores (pitch % 4 == 0, 16-byte aligned planes); a ragged
// row end takes the scalar path.  Grid: x over the 4-pixel groups of a row,
// y over rows (striding when H exceeds the grid's y limit), so no thread
// divides to find its pixel.  in == out is allowed: a thread reads all three
// channels of its pixels before it writes any.
#include <cuda_runtime.h>

#include <cstdint>

#include "bf.h"
#include "bf_internal.cuh"

namespace {

struct Mat3 {
    float m[9];
};

// IEC 61966-2-1 linear sRGB -> XYZ (D65), rows X, Y, Z.
constexpr double kRgbToXyz[9] = {0.4124, 0.3576, 0.1805, 0.2126, 0.7152, 0.0722, 0.0193, 0.1192, 0.9505};

// 1 / (row sum): dividing by the white point.
constexpr double kInvWhite[3] = {1.0 / (0.4124 + 0.3576 + 0.1805), 1.0 / (0.2126 + 0.7152 + 0.0722),
                                 1.0 / (0.0193 + 0.1192 + 0.9505)};

// XYZ / white, one row per output channel (white division folded into the matrix).
Mat3 forward_matrix() {
    Mat3 M;
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) M.m[3 * i + c] = (float)(kRgbToXyz[3 * i + c] * kInvWhite[i]);
    return M;
}

// (XYZ / white) -> linear sRGB: the inverse of forward_matrix, in FP64 by the
// adjugate (cofactor) formula.
Mat3 inverse_matrix() {
    double a[9];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) a[3 * i + c] = kRgbToXyz[3 * i + c] * kInvWhite[i];
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const double c10 = a[2] * a[7] - a[1] * a[8], c11 = a[0] * a[8] - a[2] * a[6], c12 = a[1] * a[6] - a[0] * a[7];
    const double c20 = a[1] * a[5] - a[2] * a[4], c21 = a[2] * a[3] - a[0] * a[5], c22 = a[0] * a[4] - a[1] * a[3];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    const double adj[9] = {c00, c10, c20, c01, c11, c21, c02, c12, c22};  // transpose of the cofactors
    Mat3 M;
    for (int i = 0; i < 9; ++i) M.m[i] = (float)(adj[i] / det);
    return M;
}

constexpr float kDelta = 6.0f / 29.0f;
constexpr float kDelta3 = kDelta * kDelta * kDelta;
constexpr float kLinSlope = 1.0f / (3.0f * kDelta * kDelta);  // slope of the tangent segment
constexpr float kOff = 4.0f / 29.0f;

// The powers use the SFU intrinsic __powf (exp2(y log2 x)): for the arguments
// here (x in (0.008, ~2], y in {1/3, 1/2.4, 2.4}) its documented error bound
// gives a relative error of a few 1e-6, i.e. below 1e-3 on the 0..255 and Lab
// scales; the accurate powf / cbrtf made the transforms compute-bound.
__device__ __forceinline__ float lab_f(float t) { return t > kDelta3 ? __powf(t, 1.0f / 3.0f) : fmaf(t, kLinSlope, kOff); }
__device__ __forceinline__ float lab_finv(float t) { return t > kDelta ? t * t * t : (t - kOff) * (1.0f / kLinSlope); }
__device__ __forceinline__ float srgb_decode(float v) {  // 0..255 -> linear
    const float e = v * (1.0f / 255.0f);
    return e <= 0.04045f ? e * (1.0f / 12.92f) : __powf((e + 0.055f) * (1.0f / 1.055f), 2.4f);
}
__device__ __forceinline__ float srgb_encode(float u) {  // linear -> 0..255
    const float e = u <= 0.0031308f ? 12.92f * u : fmaf(1.055f, __powf(u, 1.0f / 2.4f), -0.055f);
    return 255.0f * e;
}

__device__ __forceinline__ void to_lab(const Mat3 &M, float r, float g, float b, float &L, float &A, float &B) {
    const float lr = srgb_decode(r), lg = srgb_decode(g), lb = srgb_decode(b);
    const float fx = lab_f(fmaf(M.m[0], lr, fmaf(M.m[1], lg, M.m[2] * lb)));
    const float fy = lab_f(fmaf(M.m[3], lr, fmaf(M.m[4], lg, M.m[5] * lb)));
    const float fz = lab_f(fmaf(M.m[6], lr, fmaf(M.m[7], lg, M.m[8] * lb)));
    L = fmaf(116.0f, fy, -16.0f);
    A = 500.0f * (fx - fy);
    B = 200.0f * (fy - fz);
}

__device__ __forceinline__ void to_rgb(const Mat3 &Mi, float L, float A, float B, float &r, float &g, float &b) {
    const float fy = (L + 16.0f) * (1.0f / 116.0f);
    const float x = lab_finv(fmaf(A, 1.0f / 500.0f, fy)), y = lab_finv(fy), z = lab_finv(fmaf(-B, 1.0f / 200.0f, fy));
    r = srgb_encode(fmaf(Mi.m[0], x, fmaf(Mi.m[1], y, Mi.m[2] * z)));
    g = srgb_encode(fmaf(Mi.m[3], x, fmaf(Mi.m[4], y, Mi.m[5] * z)));
    b = srgb_encode(fmaf(Mi.m[6], x, fmaf(Mi.m[7], y, Mi.m[8] * z)));
}

template <bool TO_LAB>
__global__ void __launch_bounds__(128) color_kernel(const float *in, float *out, int H, int W, int pitch, Mat3 M) {
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= W) return;
    const size_t plane = (size_t)H * pitch;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const size_t o = (size_t)y * pitch + x;
        if (x + 4 <= W) {
            const float4 a = __ldcs(reinterpret_cast<const float4 *>(in + o));
            const float4 b = __ldcs(reinterpret_cast<const float4 *>(in + plane + o));
            const float4 c = __ldcs(reinterpret_cast<const float4 *>(in + 2 * plane + o));
            float4 p, q, s;
            if (TO_LAB) {
                to_lab(M, a.x, b.x, c.x, p.x, q.x, s.x);
                to_lab(M, a.y, b.y, c.y, p.y, q.y, s.y);
                to_lab(M, a.z, b.z, c.z, p.z, q.z, s.z);
                to_lab(M, a.w, b.w, c.w, p.w, q.w, s.w);
            } else {
                to_rgb(M, a.x, b.x, c.x, p.x, q.x, s.x);
                to_rgb(M, a.y, b.y, c.y, p.y, q.y, s.y);
                to_rgb(M, a.z, b.z, c.z, p.z, q.z, s.z);
                to_rgb(M, a.w, b.w, c.w, p.w, q.w, s.w);
            }
            __stcs(reinterpret_cast<float4 *>(out + o), p);
            __stcs(reinterpret_cast<float4 *>(out + plane + o), q);
            __stcs(reinterpret_cast<float4 *>(out + 2 * plane + o), s);
        } else {
            for (int j = x; j < W; ++j) {
                const size_t oj = (size_t)y * pitch + j;
                const float a = in[oj], b = in[plane + oj], c = in[2 * plane + oj];
                float p, q, s;
                if (TO_LAB)
                    to_lab(M, a, b, c, p, q, s);
                else
                    to_rgb(M, a, b, c, p, q, s);
                out[oj] = p;
                out[plane + oj] = q;
                out[2 * plane + oj] = s;
            }
        }
    }
}

int launch_color(bool to_lab_dir, const float *in, float *out, int H, int W, int pitch, void *stream) {
    if (H < 0 || W < 0) return BF_ERR_ARG;
    if (H == 0 || W == 0) return BF_OK;
    if (!in || !out || pitch < W) return BF_ERR_ARG;
    if ((pitch & 3) != 0 || ((uintptr_t)in & 15) != 0 || ((uintptr_t)out & 15) != 0) return BF_ERR_ALIGN;
    const size_t bytes = (size_t)3 * H * (size_t)pitch * sizeof(float);
    const char *a = (const char *)in, *b = (const char *)out;
    if (a != b && a < b + bytes && b < a + bytes) return BF_ERR_ARG;  // partial overlap
    const unsigned gx = (unsigned)(((W + 3) / 4 + 127) / 128);
    const dim3 grid(gx, (unsigned)(H < 65535 ? H : 65535));
    cudaStream_t s = (cudaStream_t)stream;
    if (to_lab_dir)
        color_kernel<true><<<grid, 128, 0, s>>>(in, out, H, W, pitch, forward_matrix());
    else
        color_kernel<false><<<grid, 128, 0, s>>>(in, out, H, W, pitch, inverse_matrix());
    return bf::cuda_err(cudaGetLastError());
}

}  // namespace

extern "C" int bf_rgb_to_lab(const float *in, float *out, int H, int W, int pitch, void *stream) {
    return launch_color(true, in, out, H, W, pitch, stream);
}

extern "C" int bf_lab_to_rgb(const float *in, float *out, int H, int W, int pitch, void *stream) {
    return launch_color(false, in, out, H, W, pitch, stream);
}
