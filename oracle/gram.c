/*
 * Oracle kernel matrix in plain C, FP64 -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's shared object. The CUDA library never links or calls it.
 *
 * Computes out[i*nb + j] = K(a_i, b_j) straight from the kernel's definition.
 * The problem statement (Sec. 1, "Problem statement") defines a kernel as a
 * function realised by inner products. The concrete kernels are these:
 *   kind 0  Gaussian   K = exp(-||a-b||^2 / param)      (Sec. 6: param = kappa)
 *   kind 1  Laplacian  K = exp(-||a-b||_2 / param)      (named in Sec. 1; the
 *                                                        paper prints no formula)
 *   kind 2  linear     K = <a,b>
 *   kind 3  polynomial K = (<a,b> + coef0)^degree
 * The squared distance is the sum of squared coordinate differences. It is
 * never the ||a||^2 + ||b||^2 - 2<a,b> expansion. One thread computes each
 * output element with no reduction across threads, so the result does not
 * depend on the thread count.
 */
#include <math.h>
#include <stdint.h>

static double kernel_value(const double* a, const double* b, int d, int kind,
                           double param, double coef0, int degree) {
  if (kind == 0 || kind == 1) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
      double diff = a[t] - b[t];
      s += diff * diff;
    }
    if (kind == 0) return exp(-s / param);
    return exp(-sqrt(s) / param);
  }
  double dot = 0.0;
  for (int t = 0; t < d; ++t) dot += a[t] * b[t];
  if (kind == 2) return dot;
  double base = dot + coef0, r = 1.0;
  for (int p = 0; p < degree; ++p) r *= base;
  return r;
}

/* Full na x nb kernel matrix between the rows of A (na x d) and B (nb x d). */
int oracle_kernel_matrix(const double* A, int64_t na, const double* B, int64_t nb,
                         int d, int kind, double param, double coef0, int degree,
                         double* out) {
  if (kind < 0 || kind > 3 || d < 0 || na < 0 || nb < 0) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < na; ++i)
    for (int64_t j = 0; j < nb; ++j)
      out[i * nb + j] = kernel_value(A + i * d, B + j * d, d, kind, param, coef0, degree);
  return 0;
}

/* Weighted kernel sums: out[i] = sum_j w[j] * K(a_i, b_j), summed in j order. */
int oracle_kernel_wsum(const double* A, int64_t na, const double* B, int64_t nb,
                       const double* w, int d, int kind, double param, double coef0,
                       int degree, double* out) {
  if (kind < 0 || kind > 3 || d < 0 || na < 0 || nb < 0) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < na; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < nb; ++j)
      s += w[j] * kernel_value(A + i * d, B + j * d, d, kind, param, coef0, degree);
    out[i] = s;
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets the number of threads later calls use (a timing knob; the results do
 * not depend on it, as no reduction crosses threads). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
