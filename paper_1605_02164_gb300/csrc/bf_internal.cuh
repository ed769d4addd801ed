// Internal declarations shared by the libbf translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "bf.h"

struct bf_plan_s {
    int d = 0, K = 0, N = 0, r = 0, whiten = 0;
    double sigma_s = 0.0;
    uint64_t seed = 0;
    int device = 0;
    // device arrays (one allocation, `block`)
    void *block = nullptr;
    bool pooled = false;       // block came from the library's stream-ordered plan pool
    float *nu_hi = nullptr;    // K*d: leading FP32 part of nu_t (turns)
    float *nu_lo = nullptr;    // K*d: FP32 remainder, nu = hi + lo to ~2^-48 relative
    double *nu64 = nullptr;    // K*d: FP64 nu_t
    int32_t *Y = nullptr;      // K*d
    float *taps = nullptr;     // taps_len floats: normalised 1-D Gaussian w(u - r), zero padded
    uint16_t *taps16 = nullptr;  // FP16 copy of the taps (tensor-core variant), taps_len
    uint16_t *tapsbf = nullptr;  // BF16 copy of the taps, taps_len
    int taps_len = 0;
    // host copies
    std::vector<int32_t> Y_host;
    std::vector<double> nu_host;
};

namespace bf {

constexpr uint32_t kPlanMagic = 0xBF1605u;

// Status word: one per device, written by device guards, read by bf_last_status.
int *status_word(int device);
// Consumes the armed one-shot fault(s) in `mask` (bf_debug_inject); true if one was armed.
bool take_fault(int mask);
// Status word of bf_filter_batch_noalloc on the current device (cleared when read).
int noalloc_take_status();

// Host-side checks shared by the image entry points (BF_OK or a BF_ERR_* code).
int check_image_args(const bf_plan_s *p, const float *in, const float *out, int H, int W, int pitch);

// FP32 fused kernel (csrc/bf_fp32.cu).
// alone: the image has the GPU to itself, so the tile height is fitted to the
// SMs; images launched side by side (the batch) keep the tallest tile.
int launch_fp32(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, cudaStream_t s,
                bool alone = true);
// Algorithm 1 with the recursive (Deriche) blur, FP32; scratch from stream_scratch.
int launch_recursive(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, cudaStream_t s);

// Tensor-core fused kernel (csrc/bf_tc.cu); variant BF_FP16TC or BF_BF16TC.
int launch_tc(const bf_plan_s &p, const float *in, float *out, int H, int W, int pitch, int variant,
              cudaStream_t s);
// One persistent launch over all tiles of n images (d = 3).  `scratch` holds
// tc_scratch_bytes(n) bytes of device memory used only by this launch's stream.
size_t tc_scratch_bytes(int n);
int tc_launch_batch(const bf_item *items, int n, int variant, void *scratch, int *status, cudaStream_t s);

// Tuned tile height (output rows) for an image of H x W in `context`
// (BF_TUNE_ALONE / BF_TUNE_BATCH), or 0 when the table has no entry (bf_tune.cu).
int tune_rows(int variant, int d, int r, int H, int W, int context);

// Library-owned device scratch for work issued on `stream`, at least `bytes`
// long (grown on demand; calls on one stream are ordered, so they may share it).
void *stream_scratch(cudaStream_t stream, size_t bytes);

inline int cuda_err(cudaError_t e) { return e == cudaSuccess ? BF_OK : BF_ERR_CUDA; }

}  // namespace bf
