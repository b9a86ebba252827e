/* Error-free residual R0 - A X for a sparse A (CSR) and a dense X -- part of
 * the FP64 oracle, TEST INFRASTRUCTURE (only the tests, smoke() and the
 * bench's CPU legs reach it, through oracle/__init__.py).
 *
 * The same arithmetic as oracle.residual_numpy, written as plain loops so
 * that the oracle can refine the large subdomains' solves in seconds:
 * per row i and right-hand side c, starting from hi = R0[i,c], lo = 0, for
 * every stored entry a of row i in storage order,
 *   (p, pe) = TwoProduct(-a, X[col, c])   Dekker (1971), Veltkamp splitting
 *   (s, se) = TwoSum(hi, p)               Knuth, TAOCP vol. 2, Sec. 4.2.2
 *   hi = s;  lo = lo + (se + pe)
 * and the result is hi + lo (the entries of a row in storage order, the
 * right-hand sides side by side).  Compiled with -ffp-contract=off so that no
 * multiply-add is fused (the splitting relies on separately rounded
 * products); the results are then bit-identical to the numpy form.
 * Rows are independent; OpenMP shares them out.
 */
#include <stdint.h>

static const double kSplit = 134217729.0; /* 2^27 + 1 */

static void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  double t = kSplit * a;
  double ah = t - (t - a);
  double al = a - ah;
  t = kSplit * b;
  double bh = t - (t - b);
  double bl = b - bh;
  *p = x;
  *e = ((ah * bh - x) + ah * bl + al * bh) + al * bl;
}

static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bb = x - a;
  *s = x;
  *e = (a - (x - bb)) + (b - bb);
}

/* out, lo: nrows x ncols caller arrays (row-major); lo holds the low parts
 * while a row is summed.  indptr, indices, data: A in CSR. */
void oracle_residual(int64_t nrows, int64_t ncols, const int64_t *indptr, const int64_t *indices,
                     const double *data, const double *X, const double *R0, double *out, double *lo) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nrows; ++i) {
    double *hi_i = out + i * ncols, *lo_i = lo + i * ncols;
    for (int64_t c = 0; c < ncols; ++c) {
      hi_i[c] = R0[i * ncols + c];
      lo_i[c] = 0.0;
    }
    for (int64_t k = indptr[i]; k < indptr[i + 1]; ++k) {
      const double a = -data[k];
      const double *x = X + indices[k] * ncols;
      for (int64_t c = 0; c < ncols; ++c) {
        double p, pe, s, se;
        two_prod(a, x[c], &p, &pe);
        two_sum(hi_i[c], p, &s, &se);
        hi_i[c] = s;
        lo_i[c] = lo_i[c] + (se + pe);
      }
    }
    for (int64_t c = 0; c < ncols; ++c) hi_i[c] = hi_i[c] + lo_i[c];
  }
}
