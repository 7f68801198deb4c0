/*
 * Plain FP64 CPU oracle for the symmetric eigenvalue decomposition A = Q Lambda Q^T.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The CUDA product path never calls
 * it, and the two share no code: no headers, no helpers, no constants.
 *
 * Everything here is deliberately unblocked and slow, so that each routine can be
 * read against the mathematics it restates:
 *
 *   orc_house        Householder reflector H = I - tau v v^T, v0 = 1, with the
 *                    LAPACK sign choice beta = -sign(alpha) ||x|| (tau = 0 when the
 *                    part below alpha is zero).
 *   orc_sytrd_lower  One-stage Householder tridiagonalization (the "one-stage
 *                    approach" of Sec. 1), optional explicit Q with A = Q T Q^T.
 *   orc_steql        Implicit QL with Wilkinson shift on a symmetric tridiagonal
 *                    (d, e) (the "QR algorithm" family of iterative solvers, Sec. 1),
 *                    eigenvalues ascending, rotations accumulated into Z.
 *   orc_bisect       Sturm-count bisection, an independent check of orc_steql.
 *   orc_jacobi       Cyclic Jacobi on a dense matrix (brute force for tiny n).
 *   orc_sbr          Successive band reduction of Sec. 2.1.1: panel QR giving
 *                    (I - W Y^T) R, then the ZY two-sided update of Eq. 1.
 *   orc_sbr_q        Forms Q_s from the reflectors orc_sbr kept.
 *   orc_bc           Bulge chasing band -> tridiagonal (Sec. 2.1.1, Sec. 4.2): one
 *                    sweep per column, each reflector applied as a full two-sided
 *                    similarity transformation of the dense matrix.
 *
 * Parallelism: OpenMP over independent rows of O(n^2) inner loops only; every value
 * is computed by one thread in a fixed order, so results do not depend on the
 * thread count.  Compiled without -ffast-math.
 *
 * Storage: column-major, element (i, j) of a matrix with leading dimension ld is
 * M[i + j*ld].  All routines take n, b as int and return 0 on success.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#include <stddef.h>

#define EL(M, ld, i, j) (M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Householder reflector.  On entry x[0] = alpha, x[1..m-1] = the part to be
 * annihilated.  On exit x[0] = beta, x[1..m-1] = v[1..m-1] (v[0] = 1 implied) and
 * (I - tau v v^T) [alpha; x] = [beta; 0].
 * ------------------------------------------------------------------------- */
void orc_house(int m, double *x, double *tau) {
  if (m <= 1) { *tau = 0.0; return; }
  double alpha = x[0];
  double ss = 0.0;
  for (int i = 1; i < m; ++i) ss += x[i] * x[i];
  if (ss == 0.0) { *tau = 0.0; return; }
  double norm = sqrt(alpha * alpha + ss);
  double beta = (alpha >= 0.0) ? -norm : norm;
  *tau = (beta - alpha) / beta;
  double scale = 1.0 / (alpha - beta);
  for (int i = 1; i < m; ++i) x[i] *= scale;
  x[0] = beta;
}

/* Copy the lower triangle onto the upper one, so that dense routines can work on
 * a full symmetric matrix. */
static void symmetrize_lower(int n, double *A, int lda) {
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) EL(A, lda, j, i) = EL(A, lda, i, j);
}

/* Two-sided application A <- H A H of H = I - tau v v^T acting on the index range
 * [r0, r0+m) of a full symmetric n x n matrix: every row and column is touched, not
 * only the band.  w = A v restricted to rows; then
 *   H A H = A - tau (A v) v^T - tau v (A v)^T + tau^2 (v^T A v) v v^T. */
static void apply_two_sided_full(int n, double *A, int lda, int r0, int m, const double *v, double tau,
                                 double *work) {
  if (tau == 0.0) return;
  /* p = A(:, r0:r0+m) v  (length n) */
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += EL(A, lda, i, r0 + k) * v[k];
    work[i] = s;
  }
  double vAv = 0.0;
  for (int k = 0; k < m; ++k) vAv += v[k] * work[r0 + k];
  /* A <- A - tau p vhat^T - tau vhat p^T + tau^2 vAv vhat vhat^T, vhat = v embedded at r0 */
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    int jin = (j >= r0 && j < r0 + m);
    double vj = jin ? v[j - r0] : 0.0;
    double pj = work[j];
    for (int i = 0; i < n; ++i) {
      int iin = (i >= r0 && i < r0 + m);
      double vi = iin ? v[i - r0] : 0.0;
      if (!iin && !jin) continue;
      EL(A, lda, i, j) += -tau * work[i] * vj - tau * vi * pj + tau * tau * vAv * vi * vj;
    }
  }
}

/* ---------------------------------------------------------------------------
 * One-stage Householder tridiagonalization of the symmetric matrix whose lower
 * triangle is in A.  A is overwritten (full symmetric working copy).  d[0..n-1],
 * e[0..n-2] receive T; if Q != NULL it receives the n x n orthogonal matrix with
 * A_in = Q T Q^T.  Reflector j acts on indices j+1..n-1 and annihilates A(j+2:n, j).
 * ------------------------------------------------------------------------- */
int orc_sytrd_lower(int n, double *A, int lda, double *d, double *e, double *Q, int ldq) {
  if (n < 0 || lda < (n > 1 ? n : 1)) return -1;
  if (n == 0) return 0;
  symmetrize_lower(n, A, lda);
  double *V = (double *)calloc((size_t)n * (size_t)n, sizeof(double)); /* reflector j in column j */
  double *taus = (double *)calloc((size_t)n, sizeof(double));
  double *p = (double *)malloc(sizeof(double) * (size_t)n);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  if (!V || !taus || !p || !w) { free(V); free(taus); free(p); free(w); return -2; }
  for (int j = 0; j + 2 < n; ++j) {
    int m = n - j - 1;            /* reflector length, rows j+1..n-1 */
    double *v = &EL(V, n, j + 1, j);
    for (int k = 0; k < m; ++k) v[k] = EL(A, lda, j + 1 + k, j);
    double tau;
    orc_house(m, v, &tau);
    double beta = v[0];
    v[0] = 1.0;
    taus[j] = tau;
    /* column j and row j now hold beta at (j+1, j), zeros below */
    EL(A, lda, j + 1, j) = beta; EL(A, lda, j, j + 1) = beta;
    for (int k = 1; k < m; ++k) { EL(A, lda, j + 1 + k, j) = 0.0; EL(A, lda, j, j + 1 + k) = 0.0; }
    if (tau != 0.0) {
      /* trailing A2 = A(j+1:, j+1:):  p = tau A2 v,  w = p - (tau/2)(p^T v) v,
       * A2 <- A2 - v w^T - w v^T  (the symmetric rank-2 form of H A2 H) */
      int r0 = j + 1;
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += EL(A, lda, r0 + i, r0 + k) * v[k];
        p[i] = tau * s;
      }
      double pv = 0.0;
      for (int i = 0; i < m; ++i) pv += p[i] * v[i];
      for (int i = 0; i < m; ++i) w[i] = p[i] - 0.5 * tau * pv * v[i];
      #pragma omp parallel for schedule(static)
      for (int c = 0; c < m; ++c)
        for (int i = 0; i < m; ++i) EL(A, lda, r0 + i, r0 + c) -= v[i] * w[c] + w[i] * v[c];
    }
  }
  for (int j = 0; j < n; ++j) d[j] = EL(A, lda, j, j);
  for (int j = 0; j + 1 < n; ++j) e[j] = EL(A, lda, j + 1, j);
  if (Q) {
    /* Q = H_0 H_1 ... H_{n-3}; accumulate backwards: Q <- H_j Q on rows j+1.. */
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) EL(Q, ldq, i, j) = (i == j) ? 1.0 : 0.0;
    for (int j = n - 3; j >= 0; --j) {
      double tau = taus[j];
      if (tau == 0.0) continue;
      int r0 = j + 1, m = n - j - 1;
      const double *v = &EL(V, n, j + 1, j);
      #pragma omp parallel for schedule(static)
      for (int c = r0; c < n; ++c) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += v[k] * EL(Q, ldq, r0 + k, c);
        s *= tau;
        for (int k = 0; k < m; ++k) EL(Q, ldq, r0 + k, c) -= s * v[k];
      }
    }
  }
  free(V); free(taus); free(p); free(w);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Implicit QL with Wilkinson shift.  d[0..n-1] diagonal, e[0..n-2] sub-diagonal
 * (e is destroyed; it must have room for n entries).  If Z != NULL, the plane
 * rotations are applied to the columns of the n x n matrix Z (pass the identity
 * for the eigenvectors of T, or Q of orc_sytrd_lower for those of A).  On exit d
 * holds the eigenvalues ascending and the columns of Z are permuted to match.
 * Returns 0, or l+1 if eigenvalue l failed to converge in 60 iterations.
 * ------------------------------------------------------------------------- */
int orc_steql(int n, double *d, double *e, double *Z, int ldz) {
  if (n <= 0) return 0;
  e[n - 1] = 0.0;
  double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)n);
  if (!cs) return -2;
  const double eps = DBL_EPSILON / 2; /* u = 2^-53 */
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int m;
      for (m = l; m < n - 1; ++m) {
        double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) { free(cs); return l + 1; }
      /* Wilkinson shift from the leading 2x2 block at l: the eigenvalue of
       * [[d_l, e_l], [e_l, d_{l+1}]] closer to d_l. */
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      double shift = d[l] - e[l] / (g + (g >= 0.0 ? r : -r));
      /* chase: start with x = d_m - shift, then rotate planes (i, i+1) for
       * i = m-1 down to l, keeping the matrix tridiagonal */
      double s = 1.0, c = 1.0, p = 0.0;
      g = d[m] - shift;
      int nrot = 0;
      int underflow = 0;
      for (int i = m - 1; i >= l; --i) {
        double f = s * e[i];
        double bb = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) { d[i + 1] -= p; e[m] = 0.0; underflow = 1; break; }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * bb;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - bb;
        cs[2 * nrot] = c; cs[2 * nrot + 1] = s; ++nrot;
      }
      if (Z && nrot > 0) {
        /* rotation k acts on columns (i, i+1) with i = m-1-k */
        #pragma omp parallel for schedule(static)
        for (int row = 0; row < n; ++row) {
          for (int k = 0; k < nrot; ++k) {
            int i = m - 1 - k;
            double cc = cs[2 * k], ss = cs[2 * k + 1];
            double zi = EL(Z, ldz, row, i), zi1 = EL(Z, ldz, row, i + 1);
            EL(Z, ldz, row, i + 1) = ss * zi + cc * zi1;
            EL(Z, ldz, row, i) = cc * zi - ss * zi1;
          }
        }
      }
      if (underflow) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  free(cs);
  /* selection sort ascending, permuting Z's columns alike */
  for (int i = 0; i < n - 1; ++i) {
    int k = i;
    for (int j = i + 1; j < n; ++j) if (d[j] < d[k]) k = j;
    if (k != i) {
      double t = d[i]; d[i] = d[k]; d[k] = t;
      if (Z)
        for (int row = 0; row < n; ++row) {
          double tz = EL(Z, ldz, row, i); EL(Z, ldz, row, i) = EL(Z, ldz, row, k); EL(Z, ldz, row, k) = tz;
        }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Sturm count: the number of eigenvalues of T strictly less than x, from the
 * signs of the pivots of the LDL^T factorization of T - x I.
 * ------------------------------------------------------------------------- */
static int sturm_count(int n, const double *d, const double *e, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

/* Every eigenvalue of (d, e) by bisection on a Gershgorin interval, to an absolute
 * width of about 2u max(|lo|, |hi|); w ascending. */
int orc_bisect(int n, const double *d, const double *e, double *w) {
  if (n <= 0) return 0;
  double lo = d[0], hi = d[0], emax = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    if (d[i] - r < lo) lo = d[i] - r;
    if (d[i] + r > hi) hi = d[i] + r;
    if (i + 1 < n && fabs(e[i]) > emax) emax = fabs(e[i]);
  }
  double tnorm = fmax(fabs(lo), fabs(hi));
  double pivmin = DBL_MIN * fmax(1.0, emax * emax);
  double pad = 2.0 * DBL_EPSILON * tnorm * n + 2.0 * pivmin;
  lo -= pad; hi += pad;
  #pragma omp parallel for schedule(dynamic, 16)
  for (int k = 0; k < n; ++k) {
    /* eigenvalue k (0-based, ascending) is the x where count(x) passes k+1 */
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (a + b);
      if (mid <= a || mid >= b) break;
      if (b - a <= 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)) + pivmin) break;
      if (sturm_count(n, d, e, mid, pivmin) >= k + 1) b = mid; else a = mid;
    }
    w[k] = 0.5 * (a + b);
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Cyclic Jacobi on the symmetric matrix whose lower triangle is in A (A is
 * destroyed).  w ascending; V (optional, ldv) the matching eigenvectors.
 * Each rotation zeroes a_pq with t = sign(theta)/(|theta| + sqrt(theta^2 + 1)),
 * theta = (a_qq - a_pp) / (2 a_pq).
 * ------------------------------------------------------------------------- */
int orc_jacobi(int n, double *A, int lda, double *w, double *V, int ldv) {
  if (n <= 0) return 0;
  symmetrize_lower(n, A, lda);
  double *Vl = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
  if (!Vl) return -2;
  for (int i = 0; i < n; ++i) EL(Vl, n, i, i) = 1.0;
  int converged = 0;
  for (int sweep = 0; sweep < 100 && !converged; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double a = EL(A, lda, i, j);
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= (DBL_EPSILON * DBL_EPSILON / 4.0) * tot * 1e-4 || off == 0.0) { converged = 1; break; }
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = EL(A, lda, p, q);
        if (apq == 0.0) continue;
        double theta = (EL(A, lda, q, q) - EL(A, lda, p, p)) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* A <- J^T A J with J the rotation in plane (p, q) */
        for (int k = 0; k < n; ++k) {
          double akp = EL(A, lda, k, p), akq = EL(A, lda, k, q);
          EL(A, lda, k, p) = c * akp - s * akq;
          EL(A, lda, k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = EL(A, lda, p, k), aqk = EL(A, lda, q, k);
          EL(A, lda, p, k) = c * apk - s * aqk;
          EL(A, lda, q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = EL(Vl, n, k, p), vkq = EL(Vl, n, k, q);
          EL(Vl, n, k, p) = c * vkp - s * vkq;
          EL(Vl, n, k, q) = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = EL(A, lda, i, i);
  for (int i = 0; i < n - 1; ++i) {
    int k = i;
    for (int j = i + 1; j < n; ++j) if (w[j] < w[k]) k = j;
    if (k != i) {
      double t = w[i]; w[i] = w[k]; w[k] = t;
      for (int r = 0; r < n; ++r) { double tv = EL(Vl, n, r, i); EL(Vl, n, r, i) = EL(Vl, n, r, k); EL(Vl, n, r, k) = tv; }
    }
  }
  if (V)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) EL(V, ldv, i, j) = EL(Vl, n, i, j);
  free(Vl);
  return converged ? 0 : 1;
}

/* ---------------------------------------------------------------------------
 * Successive band reduction (Sec. 2.1.1, Eq. 1), band half-width b.
 *
 * For panel p (columns p*b .. p*b+b-1), the panel below the band,
 * P = A(r0:n, p*b : p*b+b) with r0 = (p+1) b, is factored by Householder QR:
 * QR(P) = (I - W Y^T) R with Y unit lower trapezoidal and W = Y T (T from the
 * forward accumulation H_1 ... H_k = I - Y T Y^T).  R replaces the top of the
 * panel, zeros below.  The trailing matrix A2 = A(r0:n, r0:n) is then updated
 * with Eq. 1:
 *     Z  = A2 W - 1/2 Y (W^T A2 W)
 *     A2 = A2 - Y Z^T - Z Y^T.
 * A (lower triangle on input) is overwritten by the full symmetric band matrix
 * B = Q_s^T A Q_s.  If Ys != NULL (n x n, ldy) and taus != NULL (n), reflector i of
 * panel p is stored in column p*b+i of Ys (rows r0+i.., unit diagonal written
 * explicitly, zeros elsewhere) and its tau in taus[p*b+i].
 * ------------------------------------------------------------------------- */
int orc_sbr(int n, int b, double *A, int lda, double *Ys, int ldy, double *taus) {
  if (n < 0 || b < 1 || lda < (n > 1 ? n : 1)) return -1;
  if (n == 0) return 0;
  symmetrize_lower(n, A, lda);
  if (Ys) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) EL(Ys, ldy, i, j) = 0.0;
  if (taus) for (int j = 0; j < n; ++j) taus[j] = 0.0;
  double *Y = (double *)malloc(sizeof(double) * (size_t)n * (size_t)b);
  double *T = (double *)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double *W = (double *)malloc(sizeof(double) * (size_t)n * (size_t)b);
  double *AW = (double *)malloc(sizeof(double) * (size_t)n * (size_t)b);
  double *Zm = (double *)malloc(sizeof(double) * (size_t)n * (size_t)b);
  double *M = (double *)malloc(sizeof(double) * (size_t)b * (size_t)b);
  double *tv = (double *)malloc(sizeof(double) * (size_t)b);
  if (!Y || !T || !W || !AW || !Zm || !M || !tv) {
    free(Y); free(T); free(W); free(AW); free(Zm); free(M); free(tv); return -2;
  }
  for (int p = 0;; ++p) {
    int c0 = p * b;
    int r0 = c0 + b;
    int m = n - r0;                 /* panel rows */
    if (m < 2) break;               /* nothing below the band to annihilate */
    int bw = (n - c0 < b) ? n - c0 : b;  /* panel width */
    int k = (bw < m) ? bw : m;      /* reflectors in this panel */
    /* --- panel QR (column by column) --- */
    for (int i = 0; i < k; ++i) {
      int len = m - i;
      double *x = (double *)malloc(sizeof(double) * (size_t)len);
      for (int r = 0; r < len; ++r) x[r] = EL(A, lda, r0 + i + r, c0 + i);
      double tau;
      orc_house(len, x, &tau);
      double beta = x[0];
      /* Y(:, i): zeros above row i, 1 at row i, v below */
      for (int r = 0; r < m; ++r) EL(Y, m, r, i) = 0.0;
      EL(Y, m, i, i) = 1.0;
      for (int r = 1; r < len; ++r) EL(Y, m, i + r, i) = x[r];
      tv[i] = tau;
      /* R entry and zeros in the factored column */
      EL(A, lda, r0 + i, c0 + i) = beta;
      for (int r = 1; r < len; ++r) EL(A, lda, r0 + i + r, c0 + i) = 0.0;
      /* apply H_i to the remaining panel columns */
      for (int j = i + 1; j < bw; ++j) {
        double s = 0.0;
        for (int r = 0; r < len; ++r) s += EL(Y, m, i + r, i) * EL(A, lda, r0 + i + r, c0 + j);
        s *= tau;
        for (int r = 0; r < len; ++r) EL(A, lda, r0 + i + r, c0 + j) -= s * EL(Y, m, i + r, i);
      }
      free(x);
    }
    /* mirror the reduced panel into the upper triangle */
    for (int j = c0; j < c0 + bw; ++j)
      for (int r = r0; r < n; ++r) EL(A, lda, j, r) = EL(A, lda, r, j);
    /* --- T (k x k upper triangular) with H_0 ... H_{k-1} = I - Y T Y^T --- */
    for (int j = 0; j < k; ++j) {
      for (int i = 0; i < k; ++i) EL(T, b, i, j) = 0.0;
      EL(T, b, j, j) = tv[j];
      if (tv[j] == 0.0) continue;
      /* T(0:j, j) = -tau_j T(0:j, 0:j) (Y(:, 0:j)^T y_j) */
      double *g = (double *)malloc(sizeof(double) * (size_t)(j > 0 ? j : 1));
      for (int i = 0; i < j; ++i) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += EL(Y, m, r, i) * EL(Y, m, r, j);
        g[i] = s;
      }
      for (int i = 0; i < j; ++i) {
        double s = 0.0;
        for (int l = i; l < j; ++l) s += EL(T, b, i, l) * g[l];
        EL(T, b, i, j) = -tv[j] * s;
      }
      free(g);
    }
    /* --- W = Y T --- */
    for (int j = 0; j < k; ++j)
      for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int l = 0; l <= j; ++l) s += EL(Y, m, r, l) * EL(T, b, l, j);
        EL(W, m, r, j) = s;
      }
    /* --- Eq. 1 --- */
    /* AW = A2 W */
    #pragma omp parallel for schedule(static)
    for (int r = 0; r < m; ++r)
      for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int c = 0; c < m; ++c) s += EL(A, lda, r0 + r, r0 + c) * EL(W, m, c, j);
        EL(AW, m, r, j) = s;
      }
    /* M = W^T (A2 W) */
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += EL(W, m, r, i) * EL(AW, m, r, j);
        EL(M, b, i, j) = s;
      }
    /* Z = A2 W - 1/2 Y M */
    for (int j = 0; j < k; ++j)
      for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += EL(Y, m, r, l) * EL(M, b, l, j);
        EL(Zm, m, r, j) = EL(AW, m, r, j) - 0.5 * s;
      }
    /* A2 = A2 - Y Z^T - Z Y^T */
    #pragma omp parallel for schedule(static)
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += EL(Y, m, r, l) * EL(Zm, m, c, l) + EL(Zm, m, r, l) * EL(Y, m, c, l);
        EL(A, lda, r0 + r, r0 + c) -= s;
      }
    if (Ys && taus)
      for (int i = 0; i < k; ++i) {
        for (int r = 0; r < m; ++r) EL(Ys, ldy, r0 + r, c0 + i) = EL(Y, m, r, i);
        taus[c0 + i] = tv[i];
      }
  }
  free(Y); free(T); free(W); free(AW); free(Zm); free(M); free(tv);
  return 0;
}

/* Q_s = prod_p (I - Y_p T_p Y_p^T), formed as the product of the single
 * reflectors H = I - tau y y^T stored by orc_sbr, in panel and column order:
 * Q_s = H_{0,0} H_{0,1} ... H_{1,0} ... ; A_in = Q_s B Q_s^T. */
int orc_sbr_q(int n, const double *Ys, int ldy, const double *taus, double *Q, int ldq) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) EL(Q, ldq, i, j) = (i == j) ? 1.0 : 0.0;
  /* Q <- Q H_c for c = 0..n-1 (right multiplication, generation order) */
  for (int c = 0; c < n; ++c) {
    double tau = taus[c];
    if (tau == 0.0) continue;
    const double *y = &EL(Ys, ldy, 0, c);
    #pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += EL(Q, ldq, r, i) * y[i];
      s *= tau;
      for (int i = 0; i < n; ++i) if (y[i] != 0.0) EL(Q, ldq, r, i) -= s * y[i];
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Bulge chasing (Sec. 2.1.1 and Sec. 4.2): reduces a symmetric band matrix of
 * half-width b (lower triangle in A, entries below the band ignored and treated as
 * zero) to tridiagonal T = Q_b^T B Q_b.
 *
 * Sweep j (j = 0 .. n-3) reduces column j:
 *   step 0: rows R_0 = [j+1, j+b] (clipped to n); the reflector annihilates
 *           A(j+2 : j+b, j).
 *   step k: rows R_k = [j+1+k b, j+(k+1) b]; the reflector annihilates the first
 *           column of the bulge the previous step created, A(R_k \ top, j+1+(k-1) b).
 * Each reflector H is applied as the full similarity A <- H A H (every row and
 * column of the dense matrix), which is what the method computes; the GPU kernel
 * restricts the same arithmetic to the band and the bulge.  A step with fewer than
 * two rows is skipped (nothing to annihilate).
 * d (n), e (n-1) receive T.  If Qb != NULL it receives Q_b (n x n) with
 * B = Q_b T Q_b^T.
 * ------------------------------------------------------------------------- */
int orc_bc(int n, int b, double *A, int lda, double *d, double *e, double *Qb, int ldq) {
  if (n < 0 || b < 1 || lda < (n > 1 ? n : 1)) return -1;
  if (n == 0) return 0;
  /* densify: keep the band of the lower triangle, mirror it */
  for (int j = 0; j < n; ++j)
    for (int i = j; i < n; ++i) {
      double v = (i - j <= b) ? EL(A, lda, i, j) : 0.0;
      EL(A, lda, i, j) = v;
      EL(A, lda, j, i) = v;
    }
  if (Qb)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) EL(Qb, ldq, i, j) = (i == j) ? 1.0 : 0.0;
  double *v = (double *)malloc(sizeof(double) * (size_t)(b + 1));
  double *work = (double *)malloc(sizeof(double) * (size_t)n);
  if (!v || !work) { free(v); free(work); return -2; }
  for (int j = 0; j + 2 < n; ++j) {
    for (int k = 0;; ++k) {
      int r0 = j + 1 + k * b;
      if (r0 >= n) break;
      int r1 = r0 + b - 1;
      if (r1 > n - 1) r1 = n - 1;
      int m = r1 - r0 + 1;
      if (m < 2) break;
      int col = (k == 0) ? j : j + 1 + (k - 1) * b;
      for (int i = 0; i < m; ++i) v[i] = EL(A, lda, r0 + i, col);
      double tau;
      orc_house(m, v, &tau);
      v[0] = 1.0;
      apply_two_sided_full(n, A, lda, r0, m, v, tau, work);
      if (Qb && tau != 0.0) {
        /* Q_b <- Q_b H */
        #pragma omp parallel for schedule(static)
        for (int r = 0; r < n; ++r) {
          double s = 0.0;
          for (int i = 0; i < m; ++i) s += EL(Qb, ldq, r, r0 + i) * v[i];
          s *= tau;
          for (int i = 0; i < m; ++i) EL(Qb, ldq, r, r0 + i) -= s * v[i];
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) d[i] = EL(A, lda, i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = EL(A, lda, i + 1, i);
  free(v); free(work);
  return 0;
}
