/*
 * FP64 CPU oracle for the d-dimensional complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes (Koopman & Bisseling, "Minimizing communication in the
 * multidimensional FFT"):
 *   - the 1D DFT y_k = sum_j x_j w_n^{jk}, w_n = exp(-2 pi i / n)   (Sec. 1, eq. dft)
 *   - the d-dimensional DFT Y[k] = sum_j X[j] prod_l w_{n_l}^{j_l k_l} (Sec. 1, eq. dftd)
 *     computed row-column: a 1D FFT along every axis in turn, which is
 *     exact because the multidimensional sum factorises axis by axis
 *     (Sec. 1.2, the factorisation of the d-dim sum).
 *   - the inverse: conjugated weights and the result scaled by 1/N (Sec. 1.3).
 *   - the same sums by brute force, O(N^2) (eq. dftd written out), and at
 *     chosen output points, O(N) each.
 *
 * The 1D FFT is the textbook recursive mixed-radix Cooley-Tukey split
 * (decimation in time by the smallest prime factor r of n; a prime length is
 * summed directly), i.e. the radix split of Sec. 2.1.1 (eq. radix) applied
 * with p = r at every level.
 *
 * Layout: row-major, last axis contiguous (Sec. 3); complex numbers are
 * interleaved (re, im) doubles.  Roots of unity are evaluated with cos/sin of
 * 2*pi*e/n after reducing the integer exponent e modulo n exactly.
 *
 * Threads: OpenMP over independent lines of an axis; the number of threads
 * can be set with oracle_set_threads (0 = library default).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

/* w_n^e with w_n = exp(sign * 2 pi i / n); sign = -1 forward, +1 inverse. */
static cplx root_of_unity(int64_t e, int64_t n, int sign)
{
    e %= n;
    if (e < 0) e += n;
    double a = TWO_PI * (double)e / (double)n;
    return cos(a) + (double)sign * sin(a) * I;
}

static int64_t smallest_factor(int64_t n)
{
    if (n % 2 == 0) return 2;
    for (int64_t f = 3; f * f <= n; f += 2)
        if (n % f == 0) return f;
    return n;
}

/*
 * y[a] = sum_{j<n} x[j*xs] * w_n^{ja}, for a in [n].
 * tw[e] = w_{n0}^e for the top-level length n0; w_n^e = tw[e * tstep], tstep = n0/n.
 * tmp must hold at least n values (it is only used after the sub-calls return).
 *
 * Split j = q + r*j' (q in [r], j' in [m], m = n/r):
 *   y[k + t*m] = sum_q w_n^{q(k + t m)} Yq[k],  Yq = DFT_m of x[q + r j'].
 */
static void fft_rec(int64_t n, const cplx *x, int64_t xs, cplx *y,
                    const cplx *tw, int64_t tstep, cplx *tmp)
{
    if (n == 1) {
        y[0] = x[0];
        return;
    }
    int64_t r = smallest_factor(n);
    int64_t m = n / r;
    for (int64_t q = 0; q < r; ++q)
        fft_rec(m, x + q * xs, xs * r, y + q * m, tw, tstep * r, tmp);
    for (int64_t k = 0; k < m; ++k) {
        for (int64_t q = 0; q < r; ++q) tmp[q] = y[q * m + k];
        for (int64_t t = 0; t < r; ++t) {
            int64_t a = k + t * m;
            cplx acc = 0.0;
            for (int64_t q = 0; q < r; ++q)
                acc += tw[((q * a) % n) * tstep] * tmp[q];
            y[a] = acc;
        }
    }
}

static int g_threads = 0;

void oracle_set_threads(int t) { g_threads = t < 0 ? 0 : t; }

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * In-place 1D DFT of length shape[axis] along one axis of a d-dim row-major
 * array (every line).  sign = -1 forward (w = exp(-2 pi i/n)), +1 conjugate.
 * No scaling.  Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_fft_axis(int d, const int64_t *shape, int axis, double *data, int sign)
{
    if (d < 1 || axis < 0 || axis >= d || !shape || !data) return -1;
    if (sign != -1 && sign != 1) return -1;
    int64_t n = shape[axis], outer = 1, inner = 1;
    for (int l = 0; l < axis; ++l) outer *= shape[l];
    for (int l = axis + 1; l < d; ++l) inner *= shape[l];
    if (n < 1 || outer < 1 || inner < 1) return -1;
    if (n == 1) return 0;

    cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!tw) return -1;
    for (int64_t e = 0; e < n; ++e) tw[e] = root_of_unity(e, n, sign);

    cplx *x = (cplx *)data;
    int64_t lines = outer * inner;
    int failed = 0;
#ifdef _OPENMP
    int nt = oracle_max_threads();
#pragma omp parallel num_threads(nt) reduction(| : failed)
#endif
    {
        cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n * 3);
        if (!buf) {
            failed = 1;
        } else {
            cplx *line = buf, *res = buf + n, *tmp = buf + 2 * n;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int64_t li = 0; li < lines; ++li) {
                int64_t o = li / inner, i = li % inner;
                cplx *base = x + o * n * inner + i;
                for (int64_t j = 0; j < n; ++j) line[j] = base[j * inner];
                fft_rec(n, line, 1, res, tw, 1, tmp);
                for (int64_t j = 0; j < n; ++j) base[j * inner] = res[j];
            }
            free(buf);
        }
    }
    free(tw);
    return failed ? -1 : 0;
}

static int64_t total_size(int d, const int64_t *shape)
{
    int64_t N = 1;
    for (int l = 0; l < d; ++l) {
        if (shape[l] < 1) return -1;
        N *= shape[l];
    }
    return N;
}

/*
 * y = F_{n_1} (x) ... (x) F_{n_d} applied to x (eq. dftd), row-column.
 * inverse = 0: forward; inverse = 1: conjugated weights and scale 1/N.
 * x and y may alias.
 */
int oracle_fftn(int d, const int64_t *shape, const double *x, double *y, int inverse)
{
    if (d < 1 || !shape || !x || !y) return -1;
    int64_t N = total_size(d, shape);
    if (N < 1) return -1;
    if (x != y) memcpy(y, x, sizeof(cplx) * (size_t)N);
    int sign = inverse ? 1 : -1;
    for (int l = 0; l < d; ++l)
        if (oracle_fft_axis(d, shape, l, y, sign) != 0) return -1;
    if (inverse) {
        double s = 1.0 / (double)N;
        for (int64_t i = 0; i < 2 * N; ++i) y[i] *= s;
    }
    return 0;
}

/*
 * Brute force (eq. dftd): Y[k] = sum_j X[j] w_N^{e(j,k)} with the integer
 * exponent e = sum_l (j_l k_l mod n_l) * (N / n_l)  (mod N), since
 * w_{n_l} = w_N^{N/n_l}.  O(N^2).  inverse as in oracle_fftn.
 */
int oracle_dft_bruteforce(int d, const int64_t *shape, const double *x, double *y, int inverse)
{
    if (d < 1 || d > 16 || !shape || !x || !y || x == y) return -1;
    int64_t N = total_size(d, shape);
    if (N < 1) return -1;
    int sign = inverse ? 1 : -1;
    const cplx *X = (const cplx *)x;
    cplx *Y = (cplx *)y;
    int64_t stride_w[16];
    for (int l = 0; l < d; ++l) stride_w[l] = N / shape[l];
#ifdef _OPENMP
    int nt = oracle_max_threads();
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
    for (int64_t kf = 0; kf < N; ++kf) {
        int64_t k[16], rem = kf;
        for (int l = d - 1; l >= 0; --l) {
            k[l] = rem % shape[l];
            rem /= shape[l];
        }
        cplx acc = 0.0;
        for (int64_t jf = 0; jf < N; ++jf) {
            int64_t r = jf, e = 0;
            for (int l = d - 1; l >= 0; --l) {
                int64_t jl = r % shape[l];
                r /= shape[l];
                e += ((jl * k[l]) % shape[l]) * stride_w[l];
                e %= N;
            }
            acc += X[jf] * root_of_unity(e, N, sign);
        }
        Y[kf] = inverse ? acc / (double)N : acc;
    }
    return 0;
}

/* S(l, off) = sum_{j_l} tw_l[j_l] * S(l + 1, off * n_l + j_l); S(d, off) = X[off]. */
static cplx contract(int l, int d, const int64_t *shape, int64_t off, const cplx *X,
                     cplx *const *tw)
{
    cplx acc = 0.0;
    int64_t n = shape[l];
    if (l == d - 1) {
        const cplx *row = X + off * n;
        for (int64_t j = 0; j < n; ++j) acc += tw[l][j] * row[j];
    } else {
        for (int64_t j = 0; j < n; ++j)
            acc += tw[l][j] * contract(l + 1, d, shape, off * n + j, X, tw);
    }
    return acc;
}

/*
 * Y at npts chosen output indices k (row i of ks, d entries each), each by a
 * direct O(N) sum of eq. dftd.  inverse as in oracle_fftn.
 */
int oracle_dft_points(int d, const int64_t *shape, const double *x, int64_t npts,
                      const int64_t *ks, double *y, int inverse)
{
    if (d < 1 || d > 16 || !shape || !x || !ks || !y || npts < 0) return -1;
    int64_t N = total_size(d, shape);
    if (N < 1) return -1;
    int sign = inverse ? 1 : -1;
    int failed = 0;
#ifdef _OPENMP
    int nt = oracle_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1) reduction(| : failed)
#endif
    for (int64_t pt = 0; pt < npts; ++pt) {
        cplx *tw[16];
        int ok = 1;
        for (int l = 0; l < d; ++l) tw[l] = NULL;
        for (int l = 0; l < d; ++l) {
            int64_t kl = ks[pt * d + l];
            tw[l] = (cplx *)malloc(sizeof(cplx) * (size_t)shape[l]);
            if (!tw[l] || kl < 0 || kl >= shape[l]) {
                ok = 0;
                break;
            }
            for (int64_t j = 0; j < shape[l]; ++j)
                tw[l][j] = root_of_unity((j * kl) % shape[l], shape[l], sign);
        }
        if (ok) {
            cplx v = contract(0, d, shape, 0, (const cplx *)x, tw);
            if (inverse) v /= (double)N;
            ((cplx *)y)[pt] = v;
        } else {
            failed = 1;
        }
        for (int l = 0; l < d; ++l) free(tw[l]);
    }
    return failed ? -1 : 0;
}
