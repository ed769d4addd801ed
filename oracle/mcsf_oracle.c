/*
 * Plain FP64 CPU oracle for the Monte Carlo shiftable bilateral filter of
 * vector-valued images (Ghosh & Chaudhury, "Fast Bilateral Filtering of
 * Vector-Valued Images", arXiv 1605.02164).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark load this file.  The CUDA library never
 * links, includes or calls it, and it includes nothing from the CUDA side.
 *
 * Everything is double precision and written for a reader checking it against
 * the paper, not for speed: no blocking, no fusion, no reordering beyond what
 * the paper's equations and Algorithm 1 state.  The only concession to run
 * time is an OpenMP "parallel for" over image rows, which changes no sum.
 *
 * Images are planar (d, H, W) row-major arrays of doubles: f[c*H*W + y*W + x].
 *
 * Contents (paper section / equation in brackets):
 *   orc_splitmix64        counter-based SplitMix64 (Steele, Lea & Flood 2014)
 *   orc_sample_Y          Y = N - 2X, X ~ B(N,1/2)^d          [Prop. 2, Eq. finalApproxY]
 *   orc_cholesky          C = L L^T                            [whitening reading of Eq. COB]
 *   orc_whiten            W with W C W^T = I (Cholesky or eigen) [Eq. COB]
 *   orc_freqs             omega_t = W^T Y_t / sqrt(N)          [Eq. Ht folded]
 *   orc_direct            direct filter, part A                [Eqs. BF, normal]
 *   orc_mcsf              shiftable MC filter, part B1         [Algorithm 1, Eqs. numerator, denom]
 *   orc_mcsf_pairwise     same estimator, pairwise form, B2    [Eqs. bigExp, smallExp]
 *   orc_rc_direct         raised-cosine kernel filter, part C1 [Eq. approx]
 *   orc_deriche_blur      recursive (Deriche) Gaussian blur    [Section 3, convolution in O(1)]
 *   orc_mcsf_deriche      Algorithm 1 with the recursive blur  [same]
 *   orc_mcsf_deriche_pairwise  its pairwise form with the closed-form kernel
 *   orc_rgb_to_lab,       sRGB (0..255) <-> CIE 1976 L*a*b*, the colour transform
 *   orc_lab_to_rgb        around the filter in Section 4 (Fig. 4)
 *
 * Readings of points the paper leaves open (boundary, window, real part,
 * sampling) are stated beside the code that takes them.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOT_SPD (-2)
#define ORC_ERR_NOMEM (-5)

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Random numbers.                                                          */
/* ------------------------------------------------------------------------ */

/* Output number i (0-based) of the SplitMix64 generator started at `seed`
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014): the state advances by the golden-ratio increment and each
 * output is the state passed through the published 64-bit finaliser. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int count_ones(uint64_t v) {
    int n = 0;
    while (v) {
        n += (int)(v & 1u);
        v >>= 1;
    }
    return n;
}

/* Draw X^(1..K) from B(N,1/2)^d and store Y = N - 2X (Prop. 2 and the
 * substitution before Eq. finalApproxY).  The paper does not fix a generator;
 * the reading here is: X_k is the number of ones among N fair bits, the bits
 * being the low bits of consecutive SplitMix64 words, ceil(N/64) words per
 * (t, k), drawn t-major then k.  Y is K x d, row t = Y^(t). */
int orc_sample_Y(int d, int N, int K, uint64_t seed, int32_t *Y) {
    if (d < 1 || N < 1 || K < 0 || !Y) return ORC_ERR_ARG;
    const int words = (N + 63) / 64;
    for (int t = 0; t < K; ++t) {
        for (int k = 0; k < d; ++k) {
            int X = 0;
            for (int w = 0; w < words; ++w) {
                uint64_t idx = ((uint64_t)t * (uint64_t)d + (uint64_t)k) * (uint64_t)words + (uint64_t)w;
                uint64_t bits = orc_splitmix64(seed, idx);
                int nb = N - 64 * w;
                if (nb < 64) bits &= ((uint64_t)1 << nb) - 1u;
                X += count_ones(bits);
            }
            Y[t * d + k] = N - 2 * X;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Whitening: a matrix W with x^T C^{-1} x = |W x|^2 (Eq. COB).             */
/* ------------------------------------------------------------------------ */

/* Cholesky factor C = L L^T, L lower triangular with positive diagonal.
 * Returns ORC_ERR_NOT_SPD when a pivot is not positive. */
int orc_cholesky(int d, const double *C, double *L) {
    if (d < 1 || !C || !L) return ORC_ERR_ARG;
    memset(L, 0, sizeof(double) * (size_t)d * (size_t)d);
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = C[i * d + j];
            for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
            if (i == j) {
                if (!(s > 0.0)) return ORC_ERR_NOT_SPD;
                L[i * d + i] = sqrt(s);
            } else {
                L[i * d + j] = s / L[j * d + j];
            }
        }
    }
    return ORC_OK;
}

/* Symmetric eigen-decomposition C = V diag(lam) V^T by cyclic Jacobi
 * rotations.  Eigenvalues come out ascending (stable for ties), and each
 * eigenvector is signed so that its entry of largest magnitude (first one on
 * ties) is positive. */
static int jacobi_eig(int d, const double *C, double *lam, double *V) {
    double A[64], Vt[64];
    for (int i = 0; i < d * d; ++i) A[i] = C[i];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Vt[i * d + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                tot += A[i * d + j] * A[i * d + j];
                if (i != j) off += A[i * d + j] * A[i * d + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < d - 1; ++p)
            for (int q = p + 1; q < d; ++q) {
                double apq = A[p * d + q];
                if (apq == 0.0) continue;
                double theta = (A[q * d + q] - A[p * d + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < d; ++k) { /* A <- J^T A J, columns p, q */
                    double akp = A[k * d + p], akq = A[k * d + q];
                    A[k * d + p] = c * akp - s * akq;
                    A[k * d + q] = s * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) { /* rows p, q */
                    double apk = A[p * d + k], aqk = A[q * d + k];
                    A[p * d + k] = c * apk - s * aqk;
                    A[q * d + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < d; ++k) { /* V <- V J */
                    double vkp = Vt[k * d + p], vkq = Vt[k * d + q];
                    Vt[k * d + p] = c * vkp - s * vkq;
                    Vt[k * d + q] = s * vkp + c * vkq;
                }
            }
    }
    int order[8];
    for (int i = 0; i < d; ++i) order[i] = i;
    for (int i = 1; i < d; ++i) { /* stable insertion sort by eigenvalue */
        int o = order[i], j = i - 1;
        while (j >= 0 && A[order[j] * d + order[j]] > A[o * d + o]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = o;
    }
    for (int m = 0; m < d; ++m) {
        int col = order[m];
        lam[m] = A[col * d + col];
        int big = 0;
        for (int k = 1; k < d; ++k)
            if (fabs(Vt[k * d + col]) > fabs(Vt[big * d + col])) big = k;
        double sg = Vt[big * d + col] < 0.0 ? -1.0 : 1.0;
        for (int k = 0; k < d; ++k) V[k * d + m] = sg * Vt[k * d + col];
    }
    return ORC_OK;
}

/* Whitening matrix W (d x d, row-major) with W C W^T = I.
 *   mode 0 (Cholesky reading): W = L^{-1}, C = L L^T.
 *   mode 1 (the paper's Eq. COB): C^{-1} = Q diag(alpha^2) Q^T, W = diag(alpha) Q^T,
 *          i.e. g = Q^T f and alpha_k scales g_k. */
int orc_whiten(int d, const double *C, int mode, double *Wm) {
    if (d < 1 || d > 8 || !C || !Wm) return ORC_ERR_ARG;
    if (mode == 0) {
        double L[64];
        int rc = orc_cholesky(d, C, L);
        if (rc) return rc;
        /* Solve L W = I column by column (forward substitution). */
        for (int col = 0; col < d; ++col)
            for (int i = 0; i < d; ++i) {
                double s = (i == col) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) s -= L[i * d + k] * Wm[k * d + col];
                Wm[i * d + col] = s / L[i * d + i];
            }
        return ORC_OK;
    }
    if (mode == 1) {
        double lam[8], V[64];
        jacobi_eig(d, C, lam, V);
        for (int k = 0; k < d; ++k) {
            if (!(lam[k] > 0.0)) return ORC_ERR_NOT_SPD;
            double alpha = 1.0 / sqrt(lam[k]);
            for (int c = 0; c < d; ++c) Wm[k * d + c] = alpha * V[c * d + k];
        }
        return ORC_OK;
    }
    return ORC_ERR_ARG;
}

/* Frequency vectors omega_t = W^T Y_t / sqrt(N) (K x d), so that the phase
 * of Eq. Ht is theta_t(i) = sum_k Y_tk gamma_k g_k(i) = omega_t . f(i) with
 * g = W f and gamma = 1/sqrt(N) (the alpha_k live inside W). */
void orc_freqs(int d, int K, int N, const double *Wm, const int32_t *Y, double *omega) {
    double gamma = 1.0 / sqrt((double)N);
    for (int t = 0; t < K; ++t)
        for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += Wm[k * d + c] * (double)Y[t * d + k];
            omega[t * d + c] = s * gamma;
        }
}

/* ------------------------------------------------------------------------ */
/* Spatial kernel and window (Eq. kernel and the window rule of Section 1). */
/* ------------------------------------------------------------------------ */

/* omega(j) = exp(-|j|^2 / (2 sigma_s^2)) on the integer offsets of the
 * window [-r, r]^2 (the caller passes r; the paper's window [-3s, 3s]^2
 * holds the offsets with |j_x|, |j_y| <= floor(3 sigma_s)).  Neighbours that
 * fall outside the image are left out of both sums (the image domain Omega is
 * finite and the sums run over it). */
static double spatial2(int jy, int jx, double sigma_s) {
    return exp(-((double)jx * jx + (double)jy * jy) / (2.0 * sigma_s * sigma_s));
}

static double spatial1(int u, double sigma_s) {
    return exp(-((double)u * u) / (2.0 * sigma_s * sigma_s));
}

/* Gauss-Jordan inverse with partial pivoting (part A uses C^{-1} directly). */
static int invert(int d, const double *C, double *Ci) {
    double A[8 * 16];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < 2 * d; ++j)
            A[i * 2 * d + j] = (j < d) ? C[i * d + j] : ((j - d == i) ? 1.0 : 0.0);
    for (int col = 0; col < d; ++col) {
        int piv = col;
        for (int i = col + 1; i < d; ++i)
            if (fabs(A[i * 2 * d + col]) > fabs(A[piv * 2 * d + col])) piv = i;
        if (A[piv * 2 * d + col] == 0.0) return ORC_ERR_NOT_SPD;
        if (piv != col)
            for (int j = 0; j < 2 * d; ++j) {
                double tmp = A[col * 2 * d + j];
                A[col * 2 * d + j] = A[piv * 2 * d + j];
                A[piv * 2 * d + j] = tmp;
            }
        double p = A[col * 2 * d + col];
        for (int j = 0; j < 2 * d; ++j) A[col * 2 * d + j] /= p;
        for (int i = 0; i < d; ++i) {
            if (i == col) continue;
            double m = A[i * 2 * d + col];
            for (int j = 0; j < 2 * d; ++j) A[i * 2 * d + j] -= m * A[col * 2 * d + j];
        }
    }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Ci[i * d + j] = A[i * 2 * d + d + j];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Part A: the direct filter, Eqs. (BF) and (normal).                       */
/* ------------------------------------------------------------------------ */

/* B[f](i) = (1/Z(i)) sum_j omega(j) phi(f(i-j) - f(i)) f(i-j),
 * Z(i)   = sum_j omega(j) phi(f(i-j) - f(i)),  phi(x) = exp(-x^T C^{-1} x / 2).
 * out: d x H x W; Zout (may be NULL): H x W. */
int orc_direct(int d, int H, int W, const double *f, double sigma_s, int r,
               const double *C, double *out, double *Zout) {
    if (d < 1 || d > 8 || H < 0 || W < 0 || r < 0 || !(sigma_s > 0)) return ORC_ERR_ARG;
    double Ci[64];
    int rc = invert(d, C, Ci);
    if (rc) return rc;
    const size_t HW = (size_t)H * (size_t)W;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double Z = 0.0, num[8] = {0};
            double fi[8];
            for (int c = 0; c < d; ++c) fi[c] = f[c * HW + (size_t)y * W + x];
            for (int jy = -r; jy <= r; ++jy) {
                int yy = y - jy;
                if (yy < 0 || yy >= H) continue;
                for (int jx = -r; jx <= r; ++jx) {
                    int xx = x - jx;
                    if (xx < 0 || xx >= W) continue;
                    double delta[8];
                    for (int c = 0; c < d; ++c) delta[c] = f[c * HW + (size_t)yy * W + xx] - fi[c];
                    double q = 0.0;
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) q += delta[a] * Ci[a * d + b] * delta[b];
                    double wgt = spatial2(jy, jx, sigma_s) * exp(-0.5 * q);
                    Z += wgt;
                    for (int c = 0; c < d; ++c) num[c] += wgt * f[c * HW + (size_t)yy * W + xx];
                }
            }
            for (int c = 0; c < d; ++c) out[c * HW + (size_t)y * W + x] = num[c] / Z;
            if (Zout) Zout[(size_t)y * W + x] = Z;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Part B1: Algorithm 1 (MCSF), shiftable form.                             */
/* ------------------------------------------------------------------------ */

/* Gaussian convolution  out(i) = sum_j omega(j) in(i-j)  over the window,
 * restricted to i-j in Omega.  The 2-D kernel is the product of two 1-D
 * Gaussians and Omega is a rectangle, so the sum is taken as a pass along x
 * followed by a pass along y (the separability named after Eq. denom). */
static void gauss_conv(const double complex *in, double complex *tmp, double complex *out,
                       int H, int W, const double *w1, int r) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double complex s = 0.0;
            for (int u = -r; u <= r; ++u) {
                int xx = x - u;
                if (xx < 0 || xx >= W) continue;
                s += w1[u < 0 ? -u : u] * in[(size_t)y * W + xx];
            }
            tmp[(size_t)y * W + x] = s;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double complex s = 0.0;
            for (int v = -r; v <= r; ++v) {
                int yy = y - v;
                if (yy < 0 || yy >= H) continue;
                s += w1[v < 0 ? -v : v] * tmp[(size_t)yy * W + x];
            }
            out[(size_t)y * W + x] = s;
        }
}

/* Algorithm 1 in the paper's order:
 *   g(i) = W f(i)                      (line "Set g(i) = Q^T f(i)"; W carries alpha)
 *   gamma = 1/sqrt(N)
 *   P = 0, Z = 0
 *   for t: H(i) = prod_k exp(iota Y_tk gamma g_k(i))          (Eq. Ht)
 *          G(i) = H(i) f(i)
 *          Gbar = omega * G,  Hbar = omega * H                 (Gaussian convolutions)
 *          P += wt_t conj(H) Gbar,  Z += wt_t conj(H) Hbar    (Eqs. numerator, denom)
 *   S = P / Z
 * The paper divides the complex sums.  The reading here takes real parts,
 * S_c = Re P_c / Re Z: the imaginary parts have zero expectation because Y is
 * symmetric about 0, and the filter being approximated is real.  Weights wt_t default
 * to 1/K (Eq. finalApproxY); other weights let the exhaustive expectation of
 * Prop. 2 be evaluated with the same code.
 * Outputs (any may be NULL except out): out d x H x W, Pre/Pim d x H x W,
 * Zre/Zim H x W. */
int orc_mcsf(int d, int H, int W, const double *f, double sigma_s, int r,
             const double *Wm, int N, int K, const int32_t *Y, const double *weights,
             double *out, double *Pre, double *Zre, double *Pim, double *Zim) {
    if (d < 1 || d > 8 || H < 0 || W < 0 || r < 0 || N < 1 || K < 1 || !(sigma_s > 0)) return ORC_ERR_ARG;
    const size_t HW = (size_t)H * (size_t)W;
    if (HW == 0) return ORC_OK;
    double w1[1024];
    if (r > 1000) return ORC_ERR_ARG;
    for (int u = 0; u <= r; ++u) w1[u] = spatial1(u, sigma_s);
    const double gamma = 1.0 / sqrt((double)N);

    double *g = malloc(sizeof(double) * HW * d);
    double complex *Hc = malloc(sizeof(double complex) * HW);
    double complex *G = malloc(sizeof(double complex) * HW * d);
    double complex *tmp = malloc(sizeof(double complex) * HW);
    double complex *bar = malloc(sizeof(double complex) * HW);
    double complex *P = calloc(HW * d, sizeof(double complex));
    double complex *Zc = calloc(HW, sizeof(double complex));
    if (!g || !Hc || !G || !tmp || !bar || !P || !Zc) {
        free(g); free(Hc); free(G); free(tmp); free(bar); free(P); free(Zc);
        return ORC_ERR_NOMEM;
    }
    /* g = W f, pixel by pixel */
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < (long long)HW; ++p)
        for (int k = 0; k < d; ++k) {
            double s = 0.0;
            for (int c = 0; c < d; ++c) s += Wm[k * d + c] * f[c * HW + p];
            g[k * HW + p] = s;
        }
    for (int t = 0; t < K; ++t) {
        const double wt = weights ? weights[t] : 1.0 / (double)K;
#pragma omp parallel for schedule(static)
        for (long long p = 0; p < (long long)HW; ++p) {
            double complex h = 1.0;
            for (int k = 0; k < d; ++k) h *= cexp(I * ((double)Y[t * d + k] * gamma * g[k * HW + p]));
            Hc[p] = h;
            for (int c = 0; c < d; ++c) G[c * HW + p] = h * f[c * HW + p];
        }
        for (int c = 0; c < d; ++c) {
            gauss_conv(G + c * HW, tmp, bar, H, W, w1, r);
#pragma omp parallel for schedule(static)
            for (long long p = 0; p < (long long)HW; ++p) P[c * HW + p] += wt * conj(Hc[p]) * bar[p];
        }
        gauss_conv(Hc, tmp, bar, H, W, w1, r);
#pragma omp parallel for schedule(static)
        for (long long p = 0; p < (long long)HW; ++p) Zc[p] += wt * conj(Hc[p]) * bar[p];
    }
    for (size_t p = 0; p < HW; ++p) {
        for (int c = 0; c < d; ++c) {
            out[c * HW + p] = creal(P[c * HW + p]) / creal(Zc[p]);
            if (Pre) Pre[c * HW + p] = creal(P[c * HW + p]);
            if (Pim) Pim[c * HW + p] = cimag(P[c * HW + p]);
        }
        if (Zre) Zre[p] = creal(Zc[p]);
        if (Zim) Zim[p] = cimag(Zc[p]);
    }
    free(g); free(Hc); free(G); free(tmp); free(bar); free(P); free(Zc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Part B2: the same estimator in pairwise form, at listed pixels.          */
/* ------------------------------------------------------------------------ */

/* Substituting Eq. finalApproxY into Eq. redifBF before any shifting gives,
 * for each listed pixel i,
 *   P_c(i) = sum_t wt_t sum_j omega(j) Re[H_t(i)^* H_t(i-j)] f_c(i-j)
 *          = sum_t wt_t sum_j omega(j) cos(theta_t(i-j) - theta_t(i)) f_c(i-j),
 *   Z(i)   = sum_t wt_t sum_j omega(j) cos(theta_t(i-j) - theta_t(i)),
 * with theta_t(i) = gamma sum_k Y_tk (W f(i))_k.  This costs O(K r^2) per
 * pixel and uses the 2-D kernel directly, so it checks the shiftable form.
 * pix_yx: npix pairs (y, x).  out/Pre: npix x d;  Zre: npix. */
int orc_mcsf_pairwise(int d, int H, int W, const double *f, double sigma_s, int r,
                      const double *Wm, int N, int K, const int32_t *Y, const double *weights,
                      int npix, const int32_t *pix_yx, double *out, double *Pre, double *Zre) {
    if (d < 1 || d > 8 || H < 1 || W < 1 || r < 0 || N < 1 || K < 1 || !(sigma_s > 0)) return ORC_ERR_ARG;
    const size_t HW = (size_t)H * (size_t)W;
    const double gamma = 1.0 / sqrt((double)N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < npix; ++n) {
        int y = pix_yx[2 * n], x = pix_yx[2 * n + 1];
        double P[8] = {0}, Z = 0.0;
        double gi[8];
        for (int k = 0; k < d; ++k) {
            double s = 0.0;
            for (int c = 0; c < d; ++c) s += Wm[k * d + c] * f[c * HW + (size_t)y * W + x];
            gi[k] = s;
        }
        for (int jy = -r; jy <= r; ++jy) {
            int yy = y - jy;
            if (yy < 0 || yy >= H) continue;
            for (int jx = -r; jx <= r; ++jx) {
                int xx = x - jx;
                if (xx < 0 || xx >= W) continue;
                double gj[8];
                for (int k = 0; k < d; ++k) {
                    double s = 0.0;
                    for (int c = 0; c < d; ++c) s += Wm[k * d + c] * f[c * HW + (size_t)yy * W + xx];
                    gj[k] = s;
                }
                double ws = spatial2(jy, jx, sigma_s);
                double kern = 0.0; /* (1/T) sum_t Re[H_t(i)^* H_t(i-j)] */
                for (int t = 0; t < K; ++t) {
                    double dth = 0.0;
                    for (int k = 0; k < d; ++k) dth += (double)Y[t * d + k] * gamma * (gj[k] - gi[k]);
                    kern += (weights ? weights[t] : 1.0 / (double)K) * cos(dth);
                }
                Z += ws * kern;
                for (int c = 0; c < d; ++c) P[c] += ws * kern * f[c * HW + (size_t)yy * W + xx];
            }
        }
        for (int c = 0; c < d; ++c) {
            out[n * d + c] = P[c] / Z;
            if (Pre) Pre[n * d + c] = P[c];
        }
        if (Zre) Zre[n] = Z;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Part C1: direct filter with the order-N raised-cosine kernel, Eq. approx. */
/* ------------------------------------------------------------------------ */

static double ipow(double b, int n) {
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= b;
    return r;
}

/* psi_N(y) = prod_k cos^N(alpha_k y_k / sqrt(N)) with y the whitened
 * difference; in terms of W (which carries alpha):  prod_k cos^N((W D)_k / sqrt(N)),
 * D = f(i-j) - f(i).  Used as a direct range kernel in Eqs. BF/normal. */
int orc_rc_direct(int d, int H, int W, const double *f, double sigma_s, int r,
                  const double *Wm, int N, double *out, double *Zout) {
    if (d < 1 || d > 8 || H < 0 || W < 0 || r < 0 || N < 1 || !(sigma_s > 0)) return ORC_ERR_ARG;
    const size_t HW = (size_t)H * (size_t)W;
    const double sN = sqrt((double)N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double Z = 0.0, num[8] = {0};
            for (int jy = -r; jy <= r; ++jy) {
                int yy = y - jy;
                if (yy < 0 || yy >= H) continue;
                for (int jx = -r; jx <= r; ++jx) {
                    int xx = x - jx;
                    if (xx < 0 || xx >= W) continue;
                    double delta[8];
                    for (int c = 0; c < d; ++c)
                        delta[c] = f[c * HW + (size_t)yy * W + xx] - f[c * HW + (size_t)y * W + x];
                    double psi = 1.0;
                    for (int k = 0; k < d; ++k) {
                        double z = 0.0;
                        for (int c = 0; c < d; ++c) z += Wm[k * d + c] * delta[c];
                        psi *= ipow(cos(z / sN), N);
                    }
                    double wgt = spatial2(jy, jx, sigma_s) * psi;
                    Z += wgt;
                    for (int c = 0; c < d; ++c) num[c] += wgt * f[c * HW + (size_t)yy * W + xx];
                }
            }
            for (int c = 0; c < d; ++c) out[c * HW + (size_t)y * W + x] = num[c] / Z;
            if (Zout) Zout[(size_t)y * W + x] = Z;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* CIE-Lab colour transform used around the filter (Section 4, Fig. 4).     */
/* ------------------------------------------------------------------------ */

/* The paper filters House in CIE-Lab (citing Wyszecki & Stiles) without naming
 * the RGB space.  Reading: the RGB values are sRGB on the 0..255 scale
 * (IEC 61966-2-1: piecewise transfer function and its D65 RGB -> XYZ matrix,
 * given there to four decimals), the white point is the XYZ of RGB white (the
 * matrix's row sums), and L*a*b* is CIE 1976.  No clipping either way, so
 * out-of-gamut values produced by the filter survive the round trip. */
static const double SRGB_TO_XYZ[9] = {0.4124, 0.3576, 0.1805,   /* X */
                                      0.2126, 0.7152, 0.0722,   /* Y */
                                      0.0193, 0.1192, 0.9505};  /* Z */

static double srgb_decode(double v) { /* encoded 0..1 -> linear */
    return (v <= 0.04045) ? v / 12.92 : pow((v + 0.055) / 1.055, 2.4);
}
static double srgb_encode(double u) { /* linear -> encoded 0..1 */
    return (u <= 0.0031308) ? 12.92 * u : 1.055 * pow(u, 1.0 / 2.4) - 0.055;
}
/* CIE 1976 companding with delta = 6/29: cube root above delta^3, the tangent
 * line t / (3 delta^2) + 4/29 below it; lab_finv is its inverse. */
static double lab_f(double t) {
    const double dl = 6.0 / 29.0;
    return (t > dl * dl * dl) ? cbrt(t) : t / (3.0 * dl * dl) + 4.0 / 29.0;
}
static double lab_finv(double t) {
    const double dl = 6.0 / 29.0;
    return (t > dl) ? t * t * t : 3.0 * dl * dl * (t - 4.0 / 29.0);
}

/* rgb, lab: planar 3 x n (channel-major); 0..255 sRGB <-> (L*, a*, b*). */
int orc_rgb_to_lab(int n, const double *rgb, double *lab) {
    if (n < 0) return ORC_ERR_ARG;
    double white[3];
    for (int i = 0; i < 3; ++i) white[i] = SRGB_TO_XYZ[3 * i] + SRGB_TO_XYZ[3 * i + 1] + SRGB_TO_XYZ[3 * i + 2];
    for (int p = 0; p < n; ++p) {
        double lin[3], fx[3];
        for (int c = 0; c < 3; ++c) lin[c] = srgb_decode(rgb[(size_t)c * n + p] / 255.0);
        for (int i = 0; i < 3; ++i) {
            double xyz = 0.0;
            for (int c = 0; c < 3; ++c) xyz += SRGB_TO_XYZ[3 * i + c] * lin[c];
            fx[i] = lab_f(xyz / white[i]);
        }
        lab[p] = 116.0 * fx[1] - 16.0;
        lab[(size_t)n + p] = 500.0 * (fx[0] - fx[1]);
        lab[(size_t)2 * n + p] = 200.0 * (fx[1] - fx[2]);
    }
    return ORC_OK;
}

int orc_lab_to_rgb(int n, const double *lab, double *rgb) {
    if (n < 0) return ORC_ERR_ARG;
    double white[3], Minv[9];
    for (int i = 0; i < 3; ++i) white[i] = SRGB_TO_XYZ[3 * i] + SRGB_TO_XYZ[3 * i + 1] + SRGB_TO_XYZ[3 * i + 2];
    if (invert(3, SRGB_TO_XYZ, Minv) != ORC_OK) return ORC_ERR_ARG;
    for (int p = 0; p < n; ++p) {
        const double fy = (lab[p] + 16.0) / 116.0;
        const double f3[3] = {fy + lab[(size_t)n + p] / 500.0, fy, fy - lab[(size_t)2 * n + p] / 200.0};
        double xyz[3];
        for (int i = 0; i < 3; ++i) xyz[i] = white[i] * lab_finv(f3[i]);
        for (int c = 0; c < 3; ++c) {
            double u = 0.0;
            for (int i = 0; i < 3; ++i) u += Minv[3 * c + i] * xyz[i];
            rgb[(size_t)c * n + p] = 255.0 * srgb_encode(u);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Recursive (Deriche) Gaussian: the O(1)-in-sigma_s convolution the paper   */
/* names for Algorithm 1's convolution step (Section 3, citing Deriche 1993).*/
/* ------------------------------------------------------------------------ */

/* Deriche approximates the unnormalised Gaussian exp(-x^2 / 2 sigma^2), x >= 0,
 * by two damped sinusoids in x / sigma,
 *   h(x) = (a0 cos(w0 x/s) + a1 sin(w0 x/s)) e^{-b0 x/s}
 *        + (c0 cos(w1 x/s) + c1 sin(w1 x/s)) e^{-b1 x/s},
 * with his published fit a0 = 1.680, a1 = 3.735, b0 = 1.783, w0 = 0.6318,
 * c0 = -0.6803, c1 = -0.2598, b1 = 1.723, w1 = 1.997, and filters with h(|n|)
 * as the sum of a causal (n >= 0) and an anticausal (n <= -1) recursion.
 * The coefficients below come from the z-transform of each sampled term:
 *   e^{-beta n}(a cos(om n) + c sin(om n))  ->
 *   (a + (c sin om - a cos om) e^{-beta} z^-1) / (1 - 2 e^{-beta} cos om z^-1 + e^{-2 beta} z^-2),
 * summed over the two terms (numerator order 3, denominator order 4).  The
 * anticausal part is h(m), m >= 1, run backwards: numerator m_i = n_i - n_0 d_i.
 * Zero state at both ends of a line: inputs outside the image are zero, the
 * same truncation reading as the windowed filter (R5).  The infinite support
 * makes it a different filter from the 3-sigma window: this is its own
 * oracle variant. */
typedef struct {
    double n[4];  /* causal numerator n_0..n_3 */
    double m[5];  /* anticausal numerator m_1..m_4 (m[0] unused) */
    double dd[5]; /* denominator d_1..d_4 (dd[0] unused) */
} deriche_coef;

static const double DERICHE_FIT[8] = {1.680, 3.735, 1.783, 0.6318, -0.6803, -0.2598, 1.723, 1.997};

static void deriche_coefficients(double sigma, deriche_coef *k) {
    const double a0 = DERICHE_FIT[0], a1 = DERICHE_FIT[1], be0 = DERICHE_FIT[2] / sigma, om0 = DERICHE_FIT[3] / sigma;
    const double c0 = DERICHE_FIT[4], c1 = DERICHE_FIT[5], be1 = DERICHE_FIT[6] / sigma, om1 = DERICHE_FIT[7] / sigma;
    /* second-order denominators 1 + p_i1 z^-1 + p_i2 z^-2 and numerators q_i0 + q_i1 z^-1 */
    const double p01 = -2.0 * exp(-be0) * cos(om0), p02 = exp(-2.0 * be0);
    const double p11 = -2.0 * exp(-be1) * cos(om1), p12 = exp(-2.0 * be1);
    const double q00 = a0, q01 = (a1 * sin(om0) - a0 * cos(om0)) * exp(-be0);
    const double q10 = c0, q11 = (c1 * sin(om1) - c0 * cos(om1)) * exp(-be1);
    /* numerator q0 p1 + q1 p0 */
    k->n[0] = q00 + q10;
    k->n[1] = q00 * p11 + q01 + q10 * p01 + q11;
    k->n[2] = q00 * p12 + q01 * p11 + q10 * p02 + q11 * p01;
    k->n[3] = q01 * p12 + q11 * p02;
    /* denominator p0 p1 */
    k->dd[0] = 1.0;
    k->dd[1] = p01 + p11;
    k->dd[2] = p02 + p12 + p01 * p11;
    k->dd[3] = p01 * p12 + p11 * p02;
    k->dd[4] = p02 * p12;
    k->m[0] = 0.0;
    for (int i = 1; i <= 3; ++i) k->m[i] = k->n[i] - k->n[0] * k->dd[i];
    k->m[4] = -k->n[0] * k->dd[4];
}

/* out[i] = sum_j h(|i - j|) in[j] over the line (length n, element stride st):
 * causal recursion left to right plus anticausal recursion right to left. */
static void deriche_line(const double complex *in, double complex *out, int n, size_t st, const deriche_coef *k,
                         double complex *ya) {
    double complex yp[4] = {0, 0, 0, 0}, xp[3] = {0, 0, 0}; /* y(i-1..i-4), x(i-1..i-3) */
    for (int i = 0; i < n; ++i) {
        const double complex x = in[(size_t)i * st];
        const double complex y = k->n[0] * x + k->n[1] * xp[0] + k->n[2] * xp[1] + k->n[3] * xp[2] -
                                 k->dd[1] * yp[0] - k->dd[2] * yp[1] - k->dd[3] * yp[2] - k->dd[4] * yp[3];
        xp[2] = xp[1]; xp[1] = xp[0]; xp[0] = x;
        yp[3] = yp[2]; yp[2] = yp[1]; yp[1] = yp[0]; yp[0] = y;
        out[(size_t)i * st] = y;
    }
    double complex ym[4] = {0, 0, 0, 0}, xm[4] = {0, 0, 0, 0}; /* y(i+1..i+4), x(i+1..i+4) */
    for (int i = n - 1; i >= 0; --i) {
        const double complex y = k->m[1] * xm[0] + k->m[2] * xm[1] + k->m[3] * xm[2] + k->m[4] * xm[3] -
                                 k->dd[1] * ym[0] - k->dd[2] * ym[1] - k->dd[3] * ym[2] - k->dd[4] * ym[3];
        xm[3] = xm[2]; xm[2] = xm[1]; xm[1] = xm[0]; xm[0] = in[(size_t)i * st];
        ym[3] = ym[2]; ym[2] = ym[1]; ym[1] = ym[0]; ym[0] = y;
        ya[i] = y;
    }
    for (int i = 0; i < n; ++i) out[(size_t)i * st] += ya[i];
}

/* Separable 2-D recursive blur: rows, then columns. */
static int deriche_conv(const double complex *in, double complex *tmp, double complex *out, int H, int W,
                        const deriche_coef *k) {
    int fail = 0;
#pragma omp parallel
    {
        double complex *ya = malloc(sizeof(double complex) * (size_t)(H > W ? H : W));
        if (!ya) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(static)
        for (int y = 0; y < H; ++y)
            if (ya) deriche_line(in + (size_t)y * W, tmp + (size_t)y * W, W, 1, k, ya);
#pragma omp for schedule(static)
        for (int x = 0; x < W; ++x)
            if (ya) deriche_line(tmp + x, out + x, H, (size_t)W, k, ya);
        free(ya);
    }
    return fail ? ORC_ERR_NOMEM : ORC_OK;
}

/* The recursive blur of a real single-channel image (H x W). */
int orc_deriche_blur(int H, int W, const double *in, double sigma, double *out) {
    if (H < 0 || W < 0 || !(sigma > 0)) return ORC_ERR_ARG;
    const size_t HW = (size_t)H * W;
    if (HW == 0) return ORC_OK;
    deriche_coef k;
    deriche_coefficients(sigma, &k);
    double complex *a = malloc(sizeof(double complex) * HW), *t = malloc(sizeof(double complex) * HW),
                   *b = malloc(sizeof(double complex) * HW);
    int rc = (a && t && b) ? ORC_OK : ORC_ERR_NOMEM;
    if (rc == ORC_OK) {
        for (size_t p = 0; p < HW; ++p) a[p] = in[p];
        rc = deriche_conv(a, t, b, H, W, &k);
        if (rc == ORC_OK)
            for (size_t p = 0; p < HW; ++p) out[p] = creal(b[p]);
    }
    free(a); free(t); free(b);
    return rc;
}

/* Algorithm 1 with the recursive blur in place of the windowed one: the same
 * steps as orc_mcsf (g = W f, H_t, G_t, both blurred, combined with conj(H_t),
 * S = Re P / Re Z), each convolution being deriche_conv.  Outputs as orc_mcsf. */
int orc_mcsf_deriche(int d, int H, int W, const double *f, double sigma_s, const double *Wm, int N, int K,
                     const int32_t *Y, const double *weights, double *out, double *Pre, double *Zre) {
    if (d < 1 || d > 8 || H < 0 || W < 0 || N < 1 || K < 1 || !(sigma_s > 0)) return ORC_ERR_ARG;
    const size_t HW = (size_t)H * (size_t)W;
    if (HW == 0) return ORC_OK;
    deriche_coef kc;
    deriche_coefficients(sigma_s, &kc);
    const double gamma = 1.0 / sqrt((double)N);
    double *g = malloc(sizeof(double) * HW * d);
    double complex *Hc = malloc(sizeof(double complex) * HW);
    double complex *G = malloc(sizeof(double complex) * HW * d);
    double complex *tmp = malloc(sizeof(double complex) * HW);
    double complex *bar = malloc(sizeof(double complex) * HW);
    double complex *P = calloc(HW * d, sizeof(double complex));
    double complex *Zc = calloc(HW, sizeof(double complex));
    int rc = (g && Hc && G && tmp && bar && P && Zc) ? ORC_OK : ORC_ERR_NOMEM;
    if (rc == ORC_OK) {
#pragma omp parallel for schedule(static)
        for (long long p = 0; p < (long long)HW; ++p)
            for (int k = 0; k < d; ++k) {
                double s = 0.0;
                for (int c = 0; c < d; ++c) s += Wm[k * d + c] * f[c * HW + p];
                g[k * HW + p] = s;
            }
        for (int t = 0; t < K && rc == ORC_OK; ++t) {
            const double wt = weights ? weights[t] : 1.0 / (double)K;
#pragma omp parallel for schedule(static)
            for (long long p = 0; p < (long long)HW; ++p) {
                double complex h = 1.0;
                for (int k = 0; k < d; ++k) h *= cexp(I * ((double)Y[t * d + k] * gamma * g[k * HW + p]));
                Hc[p] = h;
                for (int c = 0; c < d; ++c) G[c * HW + p] = h * f[c * HW + p];
            }
            for (int c = 0; c < d && rc == ORC_OK; ++c) {
                rc = deriche_conv(G + c * HW, tmp, bar, H, W, &kc);
#pragma omp parallel for schedule(static)
                for (long long p = 0; p < (long long)HW; ++p) P[c * HW + p] += wt * conj(Hc[p]) * bar[p];
            }
            if (rc == ORC_OK) rc = deriche_conv(Hc, tmp, bar, H, W, &kc);
#pragma omp parallel for schedule(static)
            for (long long p = 0; p < (long long)HW; ++p) Zc[p] += wt * conj(Hc[p]) * bar[p];
        }
        if (rc == ORC_OK)
            for (size_t p = 0; p < HW; ++p) {
                for (int c = 0; c < d; ++c) {
                    out[c * HW + p] = creal(P[c * HW + p]) / creal(Zc[p]);
                    if (Pre) Pre[c * HW + p] = creal(P[c * HW + p]);
                }
                if (Zre) Zre[p] = creal(Zc[p]);
            }
    }
    free(g); free(Hc); free(G); free(tmp); free(bar); free(P); free(Zc);
    return rc;
}

/* Pairwise form of the same estimator with the recursive filter's 2-D kernel
 * written out: weight h(|jx|) h(|jy|), h Deriche's closed form above, over
 * every offset inside the image.  O(K H W) per pixel: tiny images only.  It
 * checks the recursion coefficients against the closed form they come from. */
int orc_mcsf_deriche_pairwise(int d, int H, int W, const double *f, double sigma_s, const double *Wm, int N, int K,
                              const int32_t *Y, int npix, const int32_t *pix_yx, double *out) {
    if (d < 1 || d > 8 || H < 1 || W < 1 || N < 1 || K < 1 || !(sigma_s > 0)) return ORC_ERR_ARG;
    const size_t HW = (size_t)H * (size_t)W;
    const double gamma = 1.0 / sqrt((double)N);
    const int L = H > W ? H : W;
    double *h = malloc(sizeof(double) * L);
    if (!h) return ORC_ERR_NOMEM;
    for (int n = 0; n < L; ++n) {
        const double x = n / sigma_s;
        h[n] = (DERICHE_FIT[0] * cos(DERICHE_FIT[3] * x) + DERICHE_FIT[1] * sin(DERICHE_FIT[3] * x)) *
                   exp(-DERICHE_FIT[2] * x) +
               (DERICHE_FIT[4] * cos(DERICHE_FIT[7] * x) + DERICHE_FIT[5] * sin(DERICHE_FIT[7] * x)) *
                   exp(-DERICHE_FIT[6] * x);
    }
    for (int q = 0; q < npix; ++q) {
        const int y = pix_yx[2 * q], x = pix_yx[2 * q + 1];
        double num[8] = {0}, Z = 0.0;
        for (int t = 0; t < K; ++t) {
            double th_i = 0.0;
            for (int k = 0; k < d; ++k) {
                double gk = 0.0;
                for (int c = 0; c < d; ++c) gk += Wm[k * d + c] * f[c * HW + (size_t)y * W + x];
                th_i += Y[t * d + k] * gamma * gk;
            }
            for (int yy = 0; yy < H; ++yy)
                for (int xx = 0; xx < W; ++xx) {
                    double th_j = 0.0;
                    for (int k = 0; k < d; ++k) {
                        double gk = 0.0;
                        for (int c = 0; c < d; ++c) gk += Wm[k * d + c] * f[c * HW + (size_t)yy * W + xx];
                        th_j += Y[t * d + k] * gamma * gk;
                    }
                    const double w = h[abs(y - yy)] * h[abs(x - xx)] * cos(th_j - th_i) / K;
                    Z += w;
                    for (int c = 0; c < d; ++c) num[c] += w * f[c * HW + (size_t)yy * W + xx];
                }
        }
        for (int c = 0; c < d; ++c) out[(size_t)q * d + c] = num[c] / Z;
    }
    free(h);
    return ORC_OK;
}
