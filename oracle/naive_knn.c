/* Brute-force cosine-distance k-NN in plain C (binary64).
 *
 * TEST INFRASTRUCTURE ONLY: a second, independent statement of the oracle's
 * definition, used to check oracle.py on tiny inputs. It is compiled with
 * -ffp-contract=off so that no product is fused into a following add.
 *
 * Definition (Sec. 4 and Sec. 4.2 of the paper; readings as in oracle.py):
 * for each query q and row x, D = sum q_i*x_i, A = sum q_i^2, B = sum x_i^2,
 * each summed for i = 0..F-1 in order; s = D / sqrt(A*B), or 0 if A or B is
 * 0; rows ranked by s descending, lower index first on equal s; d = 1 - s.
 */
#include <math.h>
#include <stdint.h>

static double sum_products(const float *a, const float *b, int f)
{
    double acc = 0.0;
    for (int i = 0; i < f; ++i) {
        double p = (double)a[i] * (double)b[i];
        acc = acc + p;
    }
    return acc;
}

double naive_cosine(const float *q, const float *x, int f)
{
    double d = sum_products(q, x, f);
    double a = sum_products(q, q, f);
    double b = sum_products(x, x, f);
    if (a == 0.0 || b == 0.0)
        return 0.0;
    return d / sqrt(a * b);
}

/* Is (s1, j1) ranked before (s2, j2)? */
static int better(double s1, int64_t j1, double s2, int64_t j2)
{
    return s1 > s2 || (s1 == s2 && j1 < j2);
}

/* x: n rows of f floats; q: nq rows of f floats; outputs idx[nq*k] (-1 when
 * k > n), dist[nq*k] (+inf when padded), score[nq*k]. */
void naive_knn(const float *x, int64_t n, int f, const float *q, int64_t nq,
               int k, int64_t *idx, double *dist, double *score)
{
    for (int64_t r = 0; r < nq; ++r) {
        int64_t *bi = idx + r * k;
        double *bs = score + r * k;
        for (int c = 0; c < k; ++c) {
            bi[c] = -1;
            bs[c] = -INFINITY;
        }
        for (int64_t j = 0; j < n; ++j) {
            double s = naive_cosine(q + r * f, x + j * f, f);
            /* insertion into the sorted list of the k best so far */
            int pos = k;
            while (pos > 0 && (bi[pos - 1] < 0 || better(s, j, bs[pos - 1], bi[pos - 1])))
                --pos;
            if (pos >= k)
                continue;
            for (int c = k - 1; c > pos; --c) {
                bi[c] = bi[c - 1];
                bs[c] = bs[c - 1];
            }
            bi[pos] = j;
            bs[pos] = s;
        }
        for (int c = 0; c < k; ++c)
            dist[r * k + c] = bi[c] < 0 ? INFINITY : 1.0 - bs[c];
    }
}
