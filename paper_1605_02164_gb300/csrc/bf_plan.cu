// Plan construction: sampling of Y (Prop. 2), whitening of C and the
// frequency vectors nu_t (Eq. COB folded into Eq. Ht), spatial taps (Eq. kernel).
//
// Sampling runs on the host (it is integer bookkeeping on K*d small draws);
// the whitening runs on the device in FP64: the Cholesky factor of C (or its
// Jacobi eigen-decomposition for the paper's own change of basis) and the
// back substitution that applies it to every Y_t.
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "bf_internal.cuh"

namespace bf {
namespace {

// SplitMix64 output number i for a given seed (Steele, Lea & Flood, OOPSLA
// 2014): state_i = seed + (i+1) * golden increment, output = finaliser(state_i).
inline uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// X ~ B(N, 1/2) as the number of ones among N fair bits; Y = N - 2X.
// Bits: ceil(N/64) consecutive SplitMix64 words per (t, k), t-major.
void sample_Y(int d, int N, int K, uint64_t seed, int32_t *Y) {
    const uint64_t words = (uint64_t)((N + 63) / 64);
    for (int t = 0; t < K; ++t)
        for (int k = 0; k < d; ++k) {
            int X = 0;
            uint64_t base = ((uint64_t)t * (uint64_t)d + (uint64_t)k) * words;
            int left = N;
            for (uint64_t w = 0; w < words; ++w, left -= 64) {
                uint64_t v = splitmix64_at(seed, base + w);
                if (left < 64) v &= (~0ull) >> (64 - left);
                X += __builtin_popcountll(v);
            }
            Y[t * d + k] = N - 2 * X;
        }
}

// ---------------------------------------------------------------------------
// Device FP64 whitening.  Thread 0 of every block factors C into shared
// memory; then each thread handles frequency vectors t.
// mode 0: C = L L^T, omega_t solves L^T omega_t = Y_t / sqrt(N)  (W = L^{-1}).
// mode 1: C = V diag(lam) V^T (cyclic Jacobi), W = diag(lam^{-1/2}) V^T,
//         omega_t = W^T Y_t / sqrt(N).
// ---------------------------------------------------------------------------
__device__ bool dev_cholesky(int d, const double *C, double *L) {
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int col = 0; col < d; ++col) {
        double diag = C[col * d + col];
        for (int k = 0; k < col; ++k) diag -= L[col * d + k] * L[col * d + k];
        if (!(diag > 0.0)) return false;
        double lcc = sqrt(diag);
        L[col * d + col] = lcc;
        for (int row = col + 1; row < d; ++row) {
            double v = C[row * d + col];
            for (int k = 0; k < col; ++k) v -= L[row * d + k] * L[col * d + k];
            L[row * d + col] = v / lcc;
        }
    }
    return true;
}

__device__ bool dev_eigen_whitening(int d, const double *C, double *Wm) {
    double A[BF_MAX_D * BF_MAX_D], V[BF_MAX_D * BF_MAX_D];
    for (int i = 0; i < d * d; ++i) {
        A[i] = C[i];
        V[i] = (i / d == i % d) ? 1.0 : 0.0;
    }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, all = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double a2 = A[i * d + j] * A[i * d + j];
                all += a2;
                if (i != j) off += a2;
            }
        if (off == 0.0 || off <= 1e-30 * all) break;
        for (int p = 0; p + 1 < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                double apq = A[p * d + q];
                if (apq == 0.0) continue;
                // rotation angle zeroing A[p][q]: tan(2phi) = 2 apq / (aqq - app)
                double tau = (A[q * d + q] - A[p * d + p]) / (2.0 * apq);
                double tn = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
                if (tau == 0.0) tn = 1.0;
                double cs = rsqrt(1.0 + tn * tn), sn = tn * cs;
                for (int k = 0; k < d; ++k) {
                    double x = A[k * d + p], y = A[k * d + q];
                    A[k * d + p] = cs * x - sn * y;
                    A[k * d + q] = sn * x + cs * y;
                }
                for (int k = 0; k < d; ++k) {
                    double x = A[p * d + k], y = A[q * d + k];
                    A[p * d + k] = cs * x - sn * y;
                    A[q * d + k] = sn * x + cs * y;
                }
                for (int k = 0; k < d; ++k) {
                    double x = V[k * d + p], y = V[k * d + q];
                    V[k * d + p] = cs * x - sn * y;
                    V[k * d + q] = sn * x + cs * y;
                }
            }
    }
    // ascending eigenvalues (stable), eigenvector sign: largest |entry| positive
    int idx[BF_MAX_D];
    for (int i = 0; i < d; ++i) idx[i] = i;
    for (int i = 1; i < d; ++i)
        for (int j = i; j > 0 && A[idx[j - 1] * d + idx[j - 1]] > A[idx[j] * d + idx[j]]; --j) {
            int tmp = idx[j];
            idx[j] = idx[j - 1];
            idx[j - 1] = tmp;
        }
    for (int m = 0; m < d; ++m) {
        int col = idx[m];
        double lam = A[col * d + col];
        if (!(lam > 0.0)) return false;
        int big = 0;
        for (int k = 1; k < d; ++k)
            if (fabs(V[k * d + col]) > fabs(V[big * d + col])) big = k;
        double sgn = V[big * d + col] < 0.0 ? -1.0 : 1.0;
        double alpha = 1.0 / sqrt(lam);
        for (int k = 0; k < d; ++k) Wm[m * d + k] = sgn * alpha * V[k * d + col];
    }
    return true;
}

__global__ void plan_freqs_kernel(int d, int K, int N, int mode, const double *__restrict__ C,
                                  const int32_t *__restrict__ Y, double *__restrict__ nu64,
                                  float *__restrict__ nu_hi, float *__restrict__ nu_lo, int *__restrict__ ok_out) {
    __shared__ double fac[BF_MAX_D * BF_MAX_D];  // L (mode 0) or W (mode 1)
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = mode == 0 ? dev_cholesky(d, C, fac) : dev_eigen_whitening(d, C, fac);
        if (blockIdx.x == 0) *ok_out = ok;
    }
    __syncthreads();
    if (!ok) return;
    const double inv_sqrtN = 1.0 / sqrt((double)N);
    const double inv_2pi = 0.15915494309189533577;  // 1 / (2 pi)
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < K; t += gridDim.x * blockDim.x) {
        double om[BF_MAX_D];
        if (mode == 0) {
            // back substitution L^T om = Y_t / sqrt(N), L lower triangular
            for (int i = d - 1; i >= 0; --i) {
                double v = (double)Y[t * d + i] * inv_sqrtN;
                for (int k = i + 1; k < d; ++k) v -= fac[k * d + i] * om[k];
                om[i] = v / fac[i * d + i];
            }
        } else {
            for (int c = 0; c < d; ++c) {
                double v = 0.0;
                for (int k = 0; k < d; ++k) v += fac[k * d + c] * (double)Y[t * d + k];
                om[c] = v * inv_sqrtN;
            }
        }
        for (int c = 0; c < d; ++c) {
            double nu = om[c] * inv_2pi;
            float hi = (float)nu;
            float lo = (float)(nu - (double)hi);
            nu64[t * d + c] = nu;
            nu_hi[t * d + c] = hi;
            nu_lo[t * d + c] = lo;
        }
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

namespace {
// Per device: one stream for plan set-up and a stream-ordered memory pool for
// plan blocks (allocation without a device-wide synchronisation; the pool
// keeps up to 256 MB of freed blocks for reuse).  Plans are made one at a time.
struct PlanRes {
    int device;
    cudaStream_t stream;
    cudaMemPool_t pool;  // null: plain cudaMalloc
};
std::mutex g_plan_mu;
std::vector<PlanRes> g_plan_res;

PlanRes *plan_res(int dev) {
    for (PlanRes &r : g_plan_res)
        if (r.device == dev) return &r;
    PlanRes r{dev, nullptr, nullptr};
    if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&r.pool, &props) == cudaSuccess) {
        uint64_t keep = 256ull << 20;
        cudaMemPoolSetAttribute(r.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
        cudaGetLastError();
        r.pool = nullptr;
    }
    g_plan_res.push_back(r);
    return &g_plan_res.back();
}

// Return a plan block to where it came from; the block is idle (the caller
// has synchronised).
cudaError_t release_block(bf_plan_s *p) {
    if (!p->block) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (p->pooled) {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        PlanRes *res = plan_res(p->device);
        e = res ? cudaFreeAsync(p->block, res->stream) : cudaErrorUnknown;
    } else {
        e = cudaFree(p->block);
    }
    p->block = nullptr;
    return e;
}
}  // namespace

int make_plan(int d, const double *C, double sigma_s, int N, int K, uint64_t seed, int whiten, int radius,
              bf_plan_t *out) {
    if (!out) return BF_ERR_ARG;
    *out = nullptr;
    if (d < 1 || d > BF_MAX_D) return BF_ERR_D_RANGE;
    if (!C) return BF_ERR_ARG;
    if (!(sigma_s > 0.0) || !isfinite(sigma_s)) return BF_ERR_ARG;
    if (N == 0) N = 10;
    if (N < 1 || N > BF_MAX_N || K < 1 || K > BF_MAX_K) return BF_ERR_ARG;
    if (whiten != BF_WHITEN_CHOLESKY && whiten != BF_WHITEN_EIGEN) return BF_ERR_ARG;
    double cmax = 0.0;
    for (int i = 0; i < d * d; ++i) {
        if (!isfinite(C[i])) return BF_ERR_ARG;
        cmax = fmax(cmax, fabs(C[i]));
    }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < i; ++j)
            if (fabs(C[i * d + j] - C[j * d + i]) > 1e-9 * cmax) return BF_ERR_ARG;
    int r = radius >= 0 ? radius : (int)floor(3.0 * sigma_s + 1e-9);
    if (r > BF_MAX_PLAN_RADIUS) return BF_ERR_UNSUPPORTED;

    if (take_fault(BF_FAULT_ALLOC)) return BF_ERR_NOMEM;
    bf_plan_s *p = new (std::nothrow) bf_plan_s;
    if (!p) return BF_ERR_NOMEM;
    p->d = d;
    p->K = K;
    p->N = N;
    p->r = r;
    p->whiten = whiten;
    p->sigma_s = sigma_s;
    p->seed = seed;
    cudaGetDevice(&p->device);
    p->taps_len = 8 * ((2 * r + 1 + 7) / 8) + 8;

    const size_t kd = (size_t)K * d;
    size_t off_hi = 0;
    size_t off_lo = align_up(off_hi + kd * sizeof(float), 256);
    size_t off_64 = align_up(off_lo + kd * sizeof(float), 256);
    size_t off_Y = align_up(off_64 + kd * sizeof(double), 256);
    size_t off_taps = align_up(off_Y + kd * sizeof(int32_t), 256);
    size_t off_t16 = align_up(off_taps + p->taps_len * sizeof(float), 256);
    size_t off_tbf = align_up(off_t16 + p->taps_len * sizeof(uint16_t), 256);
    size_t off_C = align_up(off_tbf + p->taps_len * sizeof(uint16_t), 256);
    size_t off_ok = align_up(off_C + (size_t)d * d * sizeof(double), 256);
    size_t total = off_ok + 256;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    PlanRes *res = plan_res(p->device);
    if (!res) {
        delete p;
        return BF_ERR_CUDA;
    }
    cudaStream_t s = res->stream;
    p->pooled = res->pool != nullptr;
    const cudaError_t ae = p->pooled ? cudaMallocFromPoolAsync(&p->block, total, res->pool, s)
                                     : cudaMalloc(&p->block, total);
    if (ae != cudaSuccess) {
        cudaGetLastError();
        p->block = nullptr;
        delete p;
        return BF_ERR_NOMEM;
    }
    char *b = (char *)p->block;
    p->nu_hi = (float *)(b + off_hi);
    p->nu_lo = (float *)(b + off_lo);
    p->nu64 = (double *)(b + off_64);
    p->Y = (int32_t *)(b + off_Y);
    p->taps = (float *)(b + off_taps);
    p->taps16 = (uint16_t *)(b + off_t16);
    p->tapsbf = (uint16_t *)(b + off_tbf);
    double *dC = (double *)(b + off_C);
    int *dok = (int *)(b + off_ok);

    p->Y_host.resize(kd);
    sample_Y(d, N, K, seed, p->Y_host.data());

    // normalised 1-D taps (the 2-D kernel is their outer product; the common
    // factor cancels in P / Z)
    std::vector<double> w(2 * r + 1);
    double sum = 0.0;
    for (int u = -r; u <= r; ++u) sum += (w[u + r] = exp(-(double)u * u / (2.0 * sigma_s * sigma_s)));
    std::vector<float> tf(p->taps_len, 0.0f);
    std::vector<uint16_t> th(p->taps_len, 0), tb(p->taps_len, 0);
    for (int u = 0; u <= 2 * r; ++u) {
        tf[u] = (float)(w[u] / sum);
        __half h = __float2half_rn((float)(w[u] / sum));
        __nv_bfloat16 bh = __float2bfloat16_rn((float)(w[u] / sum));
        memcpy(&th[u], &h, 2);
        memcpy(&tb[u], &bh, 2);
    }

    int rc = BF_OK;
    int ok = 0;
    rc |= cuda_err(cudaMemcpyAsync(dC, C, sizeof(double) * d * d, cudaMemcpyHostToDevice, s));
    rc |= cuda_err(cudaMemcpyAsync(p->Y, p->Y_host.data(), sizeof(int32_t) * kd, cudaMemcpyHostToDevice, s));
    rc |= cuda_err(cudaMemcpyAsync(p->taps, tf.data(), sizeof(float) * p->taps_len, cudaMemcpyHostToDevice, s));
    rc |= cuda_err(cudaMemcpyAsync(p->taps16, th.data(), 2 * p->taps_len, cudaMemcpyHostToDevice, s));
    rc |= cuda_err(cudaMemcpyAsync(p->tapsbf, tb.data(), 2 * p->taps_len, cudaMemcpyHostToDevice, s));
    if (rc == BF_OK) {
        int blocks = (K + 255) / 256;
        if (blocks > 64) blocks = 64;
        plan_freqs_kernel<<<blocks, 256, 0, s>>>(d, K, N, whiten, dC, p->Y, p->nu64, p->nu_hi, p->nu_lo, dok);
        rc = cuda_err(cudaGetLastError());
    }
    p->nu_host.resize(kd);
    if (rc == BF_OK) rc = cuda_err(cudaMemcpyAsync(&ok, dok, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (rc == BF_OK)
        rc = cuda_err(cudaMemcpyAsync(p->nu_host.data(), p->nu64, sizeof(double) * kd, cudaMemcpyDeviceToHost, s));
    if (rc == BF_OK) rc = cuda_err(cudaStreamSynchronize(s));  // the one wait: the SPD check needs the kernel
    if (rc == BF_OK && !ok) rc = BF_ERR_NOT_SPD;
    if (rc != BF_OK) {
        cudaGetLastError();
        cudaStreamSynchronize(s);
        if (p->pooled) cudaFreeAsync(p->block, s);
        else cudaFree(p->block);
        cudaGetLastError();
        delete p;
        return rc;
    }
    *out = p;
    return BF_OK;
}

}  // namespace bf

extern "C" int bf_plan_ex(int d, const double *C, double sigma_s, int N, int K, uint64_t seed, int whiten,
                          int radius, bf_plan_t *out) {
    return bf::make_plan(d, C, sigma_s, N, K, seed, whiten, radius, out);
}

extern "C" int bf_plan(int d, const double *C, double sigma_s, int N, int K, uint64_t seed, bf_plan_t *out) {
    return bf::make_plan(d, C, sigma_s, N, K, seed, BF_WHITEN_CHOLESKY, -1, out);
}

extern "C" int bf_plan_get_freqs(bf_plan_t p, double *nu_host, int32_t *Y_host) {
    if (!p) return BF_ERR_ARG;
    const size_t kd = (size_t)p->K * p->d;
    if (nu_host) memcpy(nu_host, p->nu_host.data(), kd * sizeof(double));
    if (Y_host) memcpy(Y_host, p->Y_host.data(), kd * sizeof(int32_t));
    return BF_OK;
}

extern "C" int bf_plan_info(bf_plan_t p, int *d, int *K, int *N, int *radius, double *sigma_s) {
    if (!p) return BF_ERR_ARG;
    if (d) *d = p->d;
    if (K) *K = p->K;
    if (N) *N = p->N;
    if (radius) *radius = p->r;
    if (sigma_s) *sigma_s = p->sigma_s;
    return BF_OK;
}

extern "C" int bf_plan_destroy(bf_plan_t p) {
    if (!p) return BF_ERR_ARG;
    // Wait for the device first, as cudaFree would: a filtering call still in
    // flight on any stream finishes before the block goes back to the pool.
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device) cudaSetDevice(p->device);
    int rc = bf::cuda_err(cudaDeviceSynchronize());
    const int rc2 = bf::cuda_err(bf::release_block(p));
    if (rc == BF_OK) rc = rc2;
    if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
    delete p;
    return rc;
}
