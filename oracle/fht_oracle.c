/*
 * fht_oracle.c -- plain, slow CPU oracle for the Brady dyadic fast Hough
 * transform (FHT) studied in Aliev, Ershov, Nikolaev, "On the use of FHT, its
 * modification for practical applications and the structure of Hough image".
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may call,
 * link or load this file. It is used by the tests, by the smoke check and by
 * the bench's CPU-baseline leg, and it shares no code with the CUDA kernels.
 *
 * Notation (the paper cites Brady for the algorithm, Section 2, and shows its
 * iterations only as a figure, Section 4 "Figure 6"; the recursion below is the
 * standard published dyadic recursion, the reading this library adopts):
 *
 *   P     n x W array, n = 2^K rows, row-major, columns taken cyclically mod W
 *   sigma +1 (shift grows to the right with y) or -1
 *   off_n(t, y) = sum_{j=1..K} bit_{K-j}(y) * ceil( floor(t / 2^(j-1)) / 2 )
 *   H[t][x]     = sum_{y<n} P[y][(x + sigma * off_n(t, y)) mod W]
 *
 *   butterfly: strips of `half` rows merge pairwise into strips of 2*half rows;
 *   in a merged strip, slope t (0 <= t < 2*half) is the top half's slope t/2 at
 *   column x plus the bottom half's slope t/2 at column x + sigma*ceil(t/2).
 *   Row s0 + t of the array holds slope t of the strip that starts at row s0.
 *
 * Every function is a direct transcription of one of those definitions: no
 * blocking, no fusion, no reordering. Floating-point variants add exactly the
 * two operands the recursion names, in IEEE round-to-nearest (build without
 * fast-math or FMA contraction).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int64_t wrap(int64_t v, int64_t m) {
    int64_t r = v % m;
    return r < 0 ? r + m : r;
}

static int ilog2_exact(int64_t n) {
    int k = 0;
    while (((int64_t)1 << k) < n) ++k;
    return k;
}

/* off_n(t, y): column offset of row y on the dyadic pattern of slope t,
 * for a strip of n = 2^K rows (closed form of the recursion above). */
int64_t fo_offset(int64_t n, int64_t t, int64_t y) {
    int K = ilog2_exact(n);
    int64_t off = 0;
    for (int j = 1; j <= K; ++j) {
        int64_t bit = (y >> (K - j)) & 1;      /* bit_{K-j}(y)              */
        int64_t q = t >> (j - 1);              /* floor(t / 2^(j-1))        */
        off += bit * ((q + 1) / 2);            /* ceil(q / 2), q >= 0       */
    }
    return off;
}

/* Brute force: H[t][x] = sum_y P[y][(x + sigma*off_n(t,y)) mod W].  O(n^2 W). */
#define DEFINE_BRUTE(T, NAME)                                                   \
    void NAME(const T *P, int n, int W, int sigma, T *H) {                      \
        for (int t = 0; t < n; ++t)                                             \
            for (int x = 0; x < W; ++x) {                                       \
                T acc = 0;                                                      \
                for (int y = 0; y < n; ++y) {                                   \
                    int64_t c = wrap(x + (int64_t)sigma * fo_offset(n, t, y), W); \
                    acc += P[(int64_t)y * W + c];                               \
                }                                                               \
                H[(int64_t)t * W + x] = acc;                                    \
            }                                                                   \
    }
DEFINE_BRUTE(int64_t, fo_brute_i64)
DEFINE_BRUTE(double, fo_brute_f64)

/* Brute-force adjoint (back-projection): out[y][c] = sum_t G[t][(c - sigma*off_n(t,y)) mod W].
 * This is the transpose of the map above, read off its definition. */
#define DEFINE_BRUTE_ADJ(T, NAME)                                               \
    void NAME(const T *G, int n, int W, int sigma, T *out) {                    \
        for (int y = 0; y < n; ++y)                                             \
            for (int c = 0; c < W; ++c) {                                       \
                T acc = 0;                                                      \
                for (int t = 0; t < n; ++t) {                                   \
                    int64_t x = wrap(c - (int64_t)sigma * fo_offset(n, t, y), W); \
                    acc += G[(int64_t)t * W + x];                               \
                }                                                               \
                out[(int64_t)y * W + c] = acc;                                  \
            }                                                                   \
    }
DEFINE_BRUTE_ADJ(int64_t, fo_brute_adjoint_i64)
DEFINE_BRUTE_ADJ(double, fo_brute_adjoint_f64)

/* Level-by-level butterfly, in place on the n x W array A. Returns 0, or -1 if
 * the scratch allocation fails. */
#define DEFINE_BUTTERFLY(T, NAME)                                               \
    int NAME(T *A, int n, int W, int sigma) {                                   \
        size_t bytes = (size_t)n * (size_t)W * sizeof(T);                       \
        T *B = (T *)malloc(bytes ? bytes : 1);                                  \
        if (!B) return -1;                                                      \
        for (int half = 1; half < n; half *= 2) {                               \
            for (int s0 = 0; s0 < n; s0 += 2 * half)                            \
                for (int t = 0; t < 2 * half; ++t) {                            \
                    const T *top = A + (int64_t)(s0 + t / 2) * W;               \
                    const T *bot = A + (int64_t)(s0 + half + t / 2) * W;        \
                    int64_t d = (int64_t)sigma * ((t + 1) / 2);                 \
                    T *out = B + (int64_t)(s0 + t) * W;                         \
                    for (int x = 0; x < W; ++x)                                 \
                        out[x] = top[x] + bot[wrap(x + d, W)];                  \
                }                                                               \
            memcpy(A, B, bytes);                                                \
        }                                                                       \
        free(B);                                                                \
        return 0;                                                               \
    }
DEFINE_BUTTERFLY(int64_t, fo_butterfly_i64)
DEFINE_BUTTERFLY(float, fo_butterfly_f32)
DEFINE_BUTTERFLY(double, fo_butterfly_f64)

/* The same recursion with another associative-commutative operation in
 * place of the sum (the paper's introduction: Hough transforms generalise to
 * any such operation): op 1 = maximum, 2 = minimum, each level taking
 * op(top[x], bot[x + sigma*ceil(t/2)]) as "top > bot ? top : bot" (max) or
 * "top < bot ? top : bot" (min). The padding stays zero (Section 3.1). */
#define DEFINE_BUTTERFLY_OP(T, NAME)                                            \
    int NAME(T *A, int n, int W, int sigma, int op) {                           \
        size_t bytes = (size_t)n * (size_t)W * sizeof(T);                       \
        T *B = (T *)malloc(bytes ? bytes : 1);                                  \
        if (!B) return -1;                                                      \
        for (int half = 1; half < n; half *= 2) {                               \
            for (int s0 = 0; s0 < n; s0 += 2 * half)                            \
                for (int t = 0; t < 2 * half; ++t) {                            \
                    const T *top = A + (int64_t)(s0 + t / 2) * W;               \
                    const T *bot = A + (int64_t)(s0 + half + t / 2) * W;        \
                    int64_t d = (int64_t)sigma * ((t + 1) / 2);                 \
                    T *out = B + (int64_t)(s0 + t) * W;                         \
                    for (int x = 0; x < W; ++x) {                               \
                        T a = top[x], b = bot[wrap(x + d, W)];                  \
                        out[x] = op == 1 ? (a > b ? a : b) : (a < b ? a : b);   \
                    }                                                           \
                }                                                               \
            memcpy(A, B, bytes);                                                \
        }                                                                       \
        free(B);                                                                \
        return 0;                                                               \
    }
DEFINE_BUTTERFLY_OP(int64_t, fo_butterfly_op_i64)
DEFINE_BUTTERFLY_OP(float, fo_butterfly_op_f32)

/* Transposed butterfly (adjoint), in place on A: levels in reverse order. In a
 * strip of 2*half rows, output slopes 2u and 2u+1 both read top row u at
 * column x and bottom row u at x + sigma*u and x + sigma*(u+1) respectively, so
 * the transpose sends g[2u] + g[2u+1] to top row u, and
 * g[2u](x - sigma*u) + g[2u+1](x - sigma*(u+1)) to bottom row u. */
#define DEFINE_ADJOINT(T, NAME)                                                 \
    int NAME(T *A, int n, int W, int sigma) {                                   \
        size_t bytes = (size_t)n * (size_t)W * sizeof(T);                       \
        T *B = (T *)malloc(bytes ? bytes : 1);                                  \
        if (!B) return -1;                                                      \
        for (int half = n / 2; half >= 1; half /= 2) {                          \
            for (int s0 = 0; s0 < n; s0 += 2 * half)                            \
                for (int u = 0; u < half; ++u) {                                \
                    const T *g0 = A + (int64_t)(s0 + 2 * u) * W;                \
                    const T *g1 = A + (int64_t)(s0 + 2 * u + 1) * W;            \
                    T *top = B + (int64_t)(s0 + u) * W;                         \
                    T *bot = B + (int64_t)(s0 + half + u) * W;                  \
                    int64_t d0 = (int64_t)sigma * u;                            \
                    int64_t d1 = (int64_t)sigma * (u + 1);                      \
                    for (int x = 0; x < W; ++x) {                               \
                        top[x] = g0[x] + g1[x];                                 \
                        bot[x] = g0[wrap(x - d0, W)] + g1[wrap(x - d1, W)];     \
                    }                                                           \
                }                                                               \
            memcpy(A, B, bytes);                                                \
        }                                                                       \
        free(B);                                                                \
        return 0;                                                               \
    }
DEFINE_ADJOINT(int64_t, fo_adjoint_i64)
DEFINE_ADJOINT(float, fo_adjoint_f32)
DEFINE_ADJOINT(double, fo_adjoint_f64)

/* Single outputs by brute force, straight from an unpadded image, for sampled
 * checks at sizes where the whole transform is too slow on the CPU.
 *
 * img      h x w image, row pitch `pitch` elements; dtype 0 = uint8,
 *          1 = int32, 2 = float32
 * transpose  nonzero: transform the transposed image (h x w is then the
 *          transposed shape; element (r, c) is read at img[c * pitch + r])
 * n, W     padded rows (power of two >= h) and cyclic width
 * For each k < count: out[k] = sum_y Pad[y][(xs[k] + sigma*off_n(ts[k], y)) mod W],
 * where Pad is the image zero-padded to n x W (zero outside h x w).
 * Integer images accumulate in int64 (returned as double, exact below 2^53). */
void fo_points(const void *img, int dtype, int h, int w, int64_t pitch, int transpose,
               int n, int W, int sigma, int count, const int64_t *ts,
               const int64_t *xs, double *out) {
    for (int k = 0; k < count; ++k) {
        int64_t iacc = 0;
        double facc = 0.0;
        for (int y = 0; y < n && y < h; ++y) {
            int64_t c = wrap(xs[k] + (int64_t)sigma * fo_offset(n, ts[k], y), W);
            if (c >= w) continue;
            int64_t idx = transpose ? c * pitch + y : (int64_t)y * pitch + c;
            if (dtype == 0) iacc += ((const uint8_t *)img)[idx];
            else if (dtype == 1) iacc += ((const int32_t *)img)[idx];
            else facc += (double)((const float *)img)[idx];
        }
        out[k] = dtype == 2 ? facc : (double)iacc;
    }
}
