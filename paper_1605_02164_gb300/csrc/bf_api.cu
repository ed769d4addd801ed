// C ABI entry points: argument checks and dispatch to the fused kernels.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "bf_internal.cuh"

namespace bf {

namespace {
std::mutex g_status_mu;
int *g_status[64] = {nullptr};

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
}  // namespace

int check_image_args(const bf_plan_s *p, const float *in, const float *out, int H, int W, int pitch) {
    if (!p) return BF_ERR_ARG;
    if (H < 0 || W < 0) return BF_ERR_ARG;
    if (H == 0 || W == 0) return BF_OK;
    if (!in || !out) return BF_ERR_ARG;
    if (pitch < W) return BF_ERR_ARG;
    if ((pitch & 3) != 0 || !aligned16(in) || !aligned16(out)) return BF_ERR_ALIGN;
    const size_t bytes = (size_t)p->d * H * (size_t)pitch * sizeof(float);
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + bytes && b < a + bytes) return BF_ERR_ARG;  // overlap
    return BF_OK;
}

std::atomic<int> g_faults{0};

bool take_fault(int mask) {
    int cur = g_faults.load();
    while (cur & mask)
        if (g_faults.compare_exchange_weak(cur, cur & ~mask)) return true;
    return false;
}

void *stream_scratch(cudaStream_t stream, size_t bytes) {
    struct Slot {
        int device;
        cudaStream_t stream;
        void *ptr;
        size_t bytes;
    };
    static std::mutex mu;
    static std::vector<Slot> slots;
    if (take_fault(BF_FAULT_ALLOC)) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    for (Slot &sl : slots)
        if (sl.device == dev && sl.stream == stream) {
            if (sl.bytes >= bytes) return sl.ptr;
            cudaStreamSynchronize(stream);  // the old buffer may still be read by queued work
            cudaFree(sl.ptr);
            sl.ptr = nullptr;
            sl.bytes = 0;
            size_t grow = std::max(bytes, (size_t)64 << 10);
            if (cudaMalloc(&sl.ptr, grow) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            sl.bytes = grow;
            return sl.ptr;
        }
    Slot sl{dev, stream, nullptr, std::max(bytes, (size_t)64 << 10)};
    if (cudaMalloc(&sl.ptr, sl.bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    slots.push_back(sl);
    return sl.ptr;
}

int *status_word(int device) {
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status[device]) {
        int *w = nullptr;
        if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        cudaMemset(w, 0, sizeof(int));
        g_status[device] = w;
    }
    return g_status[device];
}

}  // namespace bf

extern "C" int bf_filter(bf_plan_t p, const float *in, float *out, int H, int W, int pitch, int variant,
                         void *stream) {
    int rc = bf::check_image_args(p, in, out, H, W, pitch);
    if (rc != BF_OK || H == 0 || W == 0) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (variant != BF_FP32_RECURSIVE && p->r > BF_MAX_RADIUS) return BF_ERR_UNSUPPORTED;  // windowed kernels
    switch (variant) {
        case BF_FP32: return bf::launch_fp32(*p, in, out, H, W, pitch, s);
        case BF_FP16TC:
        case BF_BF16TC: return bf::launch_tc(*p, in, out, H, W, pitch, variant, s);
        case BF_FP32_RECURSIVE: return bf::launch_recursive(*p, in, out, H, W, pitch, s);
        default: return BF_ERR_ARG;
    }
}

namespace {
// Library-owned streams for the per-image FP32 launches of a batch.  A small
// image fills few of the SMs, so the images of a batch run concurrently on
// these streams; events order them after the work already queued on the
// caller's stream and before anything queued there later.
constexpr int kForks = 4;
struct Forks {
    int device = -1;
    cudaStream_t s[kForks] = {};
    cudaEvent_t start = nullptr;
    cudaEvent_t done[kForks] = {};
};
std::mutex g_fork_mu;  // also serialises the use of one device's events
std::vector<Forks> g_forks;

Forks *forks_for(int dev) {
    for (Forks &f : g_forks)
        if (f.device == dev) return &f;
    Forks f;
    f.device = dev;
    bool ok = cudaEventCreateWithFlags(&f.start, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kForks && ok; ++k)
        ok = cudaStreamCreateWithFlags(&f.s[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&f.done[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return nullptr;
    }
    g_forks.push_back(f);
    return &g_forks.back();
}

// FP32 images of a batch, spread over the fork streams and joined back.
int fp32_batch_forked(const bf_item *items, int n, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_fork_mu);
    Forks *f = forks_for(dev);
    if (!f) return BF_ERR_NOMEM;
    int rc = bf::cuda_err(cudaEventRecord(f->start, s));
    for (int k = 0; k < kForks && rc == BF_OK; ++k) rc = bf::cuda_err(cudaStreamWaitEvent(f->s[k], f->start, 0));
    if (rc != BF_OK) return rc;
    for (int i = 0, j = 0; i < n && rc == BF_OK; ++i) {
        const bf_item &it = items[i];
        if (it.H == 0 || it.W == 0) continue;
        rc = bf::launch_fp32(*it.plan, it.in, it.out, it.H, it.W, it.pitch, f->s[j++ % kForks], false);
    }
    for (int k = 0; k < kForks; ++k) {  // join even after an error, so the caller's stream stays ordered
        const int r1 = bf::cuda_err(cudaEventRecord(f->done[k], f->s[k]));
        const int r2 = bf::cuda_err(cudaStreamWaitEvent(s, f->done[k], 0));
        if (rc == BF_OK) rc = r1 != BF_OK ? r1 : r2;
    }
    return rc;
}
}  // namespace

extern "C" int bf_filter_batch(const bf_item *items, int n, int variant, void *stream) {
    if (n < 0 || (n > 0 && !items)) return BF_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        int rc = bf::check_image_args(items[i].plan, items[i].in, items[i].out, items[i].H, items[i].W,
                                      items[i].pitch);
        if (rc != BF_OK) return rc;
        if (variant != BF_FP32_RECURSIVE && items[i].plan->r > BF_MAX_RADIUS) return BF_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (variant == BF_FP16TC || variant == BF_BF16TC) {
        // every image's tiles in one persistent launch
        void *scratch = bf::stream_scratch(s, bf::tc_scratch_bytes(n));
        int dev = 0;
        cudaGetDevice(&dev);
        int *st = bf::status_word(dev);
        if (!scratch || !st) return BF_ERR_NOMEM;
        return bf::tc_launch_batch(items, n, variant, scratch, st, s);
    }
    if (variant != BF_FP32 && variant != BF_FP32_RECURSIVE) return BF_ERR_ARG;
    if (variant == BF_FP32 && n > 1) return fp32_batch_forked(items, n, s);
    for (int i = 0; i < n; ++i) {
        const bf_item &it = items[i];
        if (it.H == 0 || it.W == 0) continue;
        int rc = variant == BF_FP32 ? bf::launch_fp32(*it.plan, it.in, it.out, it.H, it.W, it.pitch, s)
                                    : bf::launch_recursive(*it.plan, it.in, it.out, it.H, it.W, it.pitch, s);
        if (rc != BF_OK) return rc;
    }
    return BF_OK;
}

namespace {
struct HostBuffers {
    std::mutex mu;
    float *dev = nullptr;
    size_t bytes = 0;
};
HostBuffers g_host;
}  // namespace

extern "C" int bf_filter_host(bf_plan_t p, const float *in_host, float *out_host, int H, int W, int variant,
                              void *stream) {
    if (!p || H < 0 || W < 0) return BF_ERR_ARG;
    if (H == 0 || W == 0) return BF_OK;
    if (!in_host || !out_host) return BF_ERR_ARG;
    const int pitch = (W + 3) & ~3;
    const size_t img = (size_t)p->d * H * (size_t)pitch * sizeof(float);
    const size_t need = 2 * ((img + 255) / 256 * 256);
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_host.mu);
    if (g_host.bytes < need) {
        if (g_host.dev) {
            cudaStreamSynchronize(s);
            cudaFree(g_host.dev);
        }
        g_host.dev = nullptr;
        g_host.bytes = 0;
        if (cudaMalloc(&g_host.dev, need) != cudaSuccess) {
            cudaGetLastError();
            return BF_ERR_NOMEM;
        }
        g_host.bytes = need;
    }
    float *din = g_host.dev;
    float *dout = (float *)((char *)g_host.dev + need / 2);
    const size_t plane_h = (size_t)H * W, plane_d = (size_t)H * pitch;
    int rc = BF_OK;
    for (int c = 0; c < p->d && rc == BF_OK; ++c)
        rc = bf::cuda_err(cudaMemcpy2DAsync(din + c * plane_d, pitch * sizeof(float), in_host + c * plane_h,
                                            W * sizeof(float), W * sizeof(float), H, cudaMemcpyHostToDevice, s));
    if (rc == BF_OK) rc = bf_filter(p, din, dout, H, W, pitch, variant, stream);
    for (int c = 0; c < p->d && rc == BF_OK; ++c)
        rc = bf::cuda_err(cudaMemcpy2DAsync(out_host + c * plane_h, W * sizeof(float), dout + c * plane_d,
                                            pitch * sizeof(float), W * sizeof(float), H, cudaMemcpyDeviceToHost, s));
    if (rc == BF_OK) rc = bf::cuda_err(cudaStreamSynchronize(s));
    return rc;
}

namespace {
// Device buffers of bf_filter_host_async: one in/out pair per (device, stream),
// grown on demand; a call is ordered after the previous one on its stream.
struct IoSlot {
    int device;
    cudaStream_t stream;
    void *ptr;
    size_t bytes;
};
std::mutex g_io_mu;
std::vector<IoSlot> g_io;

void *io_buffers(cudaStream_t s, size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_io_mu);
    IoSlot *slot = nullptr;
    for (IoSlot &sl : g_io)
        if (sl.device == dev && sl.stream == s) slot = &sl;
    if (slot && slot->bytes >= bytes) return slot->ptr;
    if (!slot) {
        g_io.push_back(IoSlot{dev, s, nullptr, 0});
        slot = &g_io.back();
    }
    if (slot->ptr) {
        cudaStreamSynchronize(s);  // queued copies may still use the old buffers
        cudaFree(slot->ptr);
        slot->ptr = nullptr;
        slot->bytes = 0;
    }
    if (cudaMalloc(&slot->ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    slot->bytes = bytes;
    return slot->ptr;
}
}  // namespace

extern "C" int bf_filter_host_async(bf_plan_t p, const float *in_host, float *out_host, int H, int W, int variant,
                                    void *stream) {
    if (!p || H < 0 || W < 0) return BF_ERR_ARG;
    if (H == 0 || W == 0) return BF_OK;
    if (!in_host || !out_host) return BF_ERR_ARG;
    const int pitch = (W + 3) & ~3;
    const size_t img = (size_t)p->d * H * (size_t)pitch * sizeof(float);
    const size_t half = (img + 255) / 256 * 256;
    cudaStream_t s = (cudaStream_t)stream;
    char *buf = (char *)io_buffers(s, 2 * half);
    if (!buf) return BF_ERR_NOMEM;
    float *din = (float *)buf, *dout = (float *)(buf + half);
    const size_t plane_h = (size_t)H * W, plane_d = (size_t)H * pitch;
    int rc = BF_OK;
    for (int c = 0; c < p->d && rc == BF_OK; ++c)
        rc = bf::cuda_err(cudaMemcpy2DAsync(din + c * plane_d, pitch * sizeof(float), in_host + c * plane_h,
                                            W * sizeof(float), W * sizeof(float), H, cudaMemcpyHostToDevice, s));
    if (rc == BF_OK) rc = bf_filter(p, din, dout, H, W, pitch, variant, stream);
    for (int c = 0; c < p->d && rc == BF_OK; ++c)
        rc = bf::cuda_err(cudaMemcpy2DAsync(out_host + c * plane_h, W * sizeof(float), dout + c * plane_d,
                                            pitch * sizeof(float), W * sizeof(float), H, cudaMemcpyDeviceToHost, s));
    return rc;
}

extern "C" int bf_last_status(void *stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BF_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BF_ERR_CUDA;
    int *w = bf::status_word(dev);
    if (!w) return BF_ERR_NOMEM;
    int v = 0;
    if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BF_ERR_CUDA;
    if (v != 0) cudaMemset(w, 0, sizeof(int));
    const int v2 = bf::noalloc_take_status();  // the allocation-free entry point keeps its own word
    return v != 0 ? v : v2;
}

extern "C" int bf_debug_inject(int faults) {
    if (faults & ~(BF_FAULT_ALLOC | BF_FAULT_TC_WAIT)) return BF_ERR_ARG;
    if (faults == 0)
        bf::g_faults.store(0);
    else
        bf::g_faults.fetch_or(faults);
    return BF_OK;
}

extern "C" const char *bf_error_string(int code) {
    switch (code) {
        case BF_OK: return "ok";
        case BF_ERR_ARG: return "invalid argument";
        case BF_ERR_NOT_SPD: return "covariance is not symmetric positive definite";
        case BF_ERR_D_RANGE: return "channel count outside [1, BF_MAX_D]";
        case BF_ERR_ALIGN: return "pointer or pitch not 16-byte aligned";
        case BF_ERR_NOMEM: return "allocation failed";
        case BF_ERR_BUDGET: return "request exceeds the memory budget";
        case BF_ERR_TIMEOUT: return "bounded device wait ran out";
        case BF_ERR_CUDA: return "CUDA runtime error";
        case BF_ERR_UNSUPPORTED: return "parameters outside the supported range";
        case BF_ERR_BOUNDS: return "device-side index check failed";
        default: return "unknown error";
    }
}

extern "C" int bf_version(void) { return 10000; }
