// Divide and conquer for the symmetric tridiagonal eigenproblem, on the device.
//
// Cuppen's method with the Gu-Eisenstat eigenvector formula (the solver the
// paper names for T -> Lambda, Q_d, Sec. 1 and Sec. 3.3):
//   * tear: T = diag(T1, T2) + rho v v^T with v = e_m + sign(beta) e_{m+1},
//     rho = |beta|, beta the coupling entry; T1's last and T2's first diagonal lose
//     |beta|.  Recursively down to leaves of at most 32 rows.
//   * leaves: implicit QL with Wilkinson shift, one warp per leaf (lane = row of
//     the leaf's eigenvector matrix).
//   * merge of (Q1, L1), (Q2, L2): z = [last row of Q1, sign(beta) first row of Q2]
//     / sqrt(2), rho = 2 |beta|; sort the poles; deflate small rho z_i and nearly
//     equal poles (Givens rotation); solve the secular equation
//     1 + rho sum z_j^2 / (d_j - lambda) = 0 for each remaining root with a
//     bracketed rational ("middle way") iteration in a shifted variable;
//     recompute z by the Loewner formula; form the eigenvectors
//     u_i = zhat / (d - lambda_i) (normalised); multiply Q_block U with the dense
//     product engine; merge-sort the eigenpairs.
// All secular-equation arithmetic is FP64.
#include <cmath>
#include <cstdio>
#include <vector>

#include "device_util.cuh"
#include "evd_internal.h"

namespace evd {

namespace {

constexpr int LEAF = 32;
constexpr double kU = 1.1102230246251565e-16;  // 2^-53

struct MergeDesc {
  int64_t off, n1, n2;
};

// ---------------------------------------------------------------- tear
__global__ void k_dc_tear(const MergeDesc* md, int count, double* d, const double* e) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const MergeDesc m = md[t];
  int64_t i = m.off + m.n1 - 1;
  double ab = fabs(e[i]);
  d[i] -= ab;
  d[i + 1] -= ab;
}

// ---------------------------------------------------------------- leaves
// One warp per leaf of size <= 32.  Lane r holds row r of the leaf's Z.
__global__ void k_dc_leaf(const int64_t* leaf_off, const int* leaf_n, int nleaves, double* d, const double* e,
                          double* Q, int64_t ldq, int* st) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nleaves) return;
  const int64_t off = leaf_off[warp];
  const int n = leaf_n[warp];
  __shared__ double sd[4][LEAF], se[4][LEAF];
  const int wl = threadIdx.x >> 5;
  double* dd = sd[wl];
  double* ee = se[wl];
  if (lane < n) {
    dd[lane] = d[off + lane];
    ee[lane] = (lane + 1 < n) ? e[off + lane] : 0.0;
  }
  __syncwarp();
  double z[LEAF];
#pragma unroll
  for (int c = 0; c < LEAF; ++c) z[c] = (c == lane) ? 1.0 : 0.0;
  // implicit QL, every lane runs the same scalar recurrence on its own copy of d/e
  double dl[LEAF], el[LEAF];
#pragma unroll
  for (int c = 0; c < LEAF; ++c) { dl[c] = (c < n) ? dd[c] : 0.0; el[c] = (c < n) ? ee[c] : 0.0; }
  bool fail = false;
  for (int l = 0; l < n && !fail; ++l) {
    int iter = 0;
    for (;;) {
      int m;
      for (m = l; m < n - 1; ++m) {
        double s = fabs(dl[m]) + fabs(dl[m + 1]);
        if (fabs(el[m]) <= kU * s) break;
      }
      if (m == l) break;
      if (++iter > 60) { fail = true; break; }
      double g = (dl[l + 1] - dl[l]) / (2.0 * el[l]);
      double r = hypot(g, 1.0);
      double shift = dl[l] - el[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      g = dl[m] - shift;
      bool under = false;
      for (int i = m - 1; i >= l; --i) {
        double f = s * el[i], bb = c * el[i];
        r = hypot(f, g);
        el[i + 1] = r;
        if (r == 0.0) { dl[i + 1] -= p; el[m] = 0.0; under = true; break; }
        s = f / r; c = g / r;
        g = dl[i + 1] - p;
        r = (dl[i] - g) * s + 2.0 * c * bb;
        p = s * r;
        dl[i + 1] = g + p;
        g = c * r - bb;
        // rotate columns i, i+1 of Z (this lane's row)
        double zi = z[i], zi1 = z[i + 1];
        z[i + 1] = s * zi + c * zi1;
        z[i] = c * zi - s * zi1;
      }
      if (under) continue;
      dl[l] -= p; el[l] = g; el[m] = 0.0;
    }
  }
  if (fail) {
    if (lane == 0) dev_set_status(st, EVD_ERR_NO_CONVERGENCE, (int)(off + 1));
    return;
  }
  // selection sort ascending, permuting Z columns
  for (int i = 0; i < n - 1; ++i) {
    int kk = i;
    for (int j = i + 1; j < n; ++j) if (dl[j] < dl[kk]) kk = j;
    if (kk != i) {
      double t = dl[i]; dl[i] = dl[kk]; dl[kk] = t;
      double tz = z[i]; z[i] = z[kk]; z[kk] = tz;
    }
  }
  if (lane < n) {
    d[off + lane] = dl[lane];
    for (int c = 0; c < n; ++c) Q[(off + lane) + (off + c) * ldq] = z[c];
  }
}

// ---------------------------------------------------------------- merge: prepare
// z, rho, merge-sort of the two pole lists.  One CTA per merge.
// Outputs at [off, off+m): ds (sorted poles), zs (z in sorted order), perm (source
// column within the block), and per merge: rho, tol.
__global__ void k_dc_prepare(const MergeDesc* md, const double* d, const double* e, const double* Q, int64_t ldq,
                             double* ds, double* zs, int* perm, double* rho_out, double* tol_out) {
  const MergeDesc M = md[blockIdx.x];
  const int64_t off = M.off, n1 = M.n1, n2 = M.n2, m = n1 + n2;
  const double beta = e[off + n1 - 1];
  const double sgn = (beta >= 0.0) ? 1.0 : -1.0;
  const double isq2 = 0.70710678118654752440;
  __shared__ double red[256];
  double dmax = 0.0;
  for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
    double dv, zv;
    int64_t rank;
    if (t < n1) {
      dv = d[off + t];
      zv = Q[(off + n1 - 1) + (off + t) * ldq] * isq2;
      // rank: t + #{elements of list 2 strictly less than dv}
      int64_t lo = 0, hi = n2;
      while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (d[off + n1 + mid] < dv) lo = mid + 1; else hi = mid; }
      rank = t + lo;
    } else {
      int64_t u = t - n1;
      dv = d[off + t];
      zv = sgn * Q[(off + n1) + (off + t) * ldq] * isq2;
      // rank: u + #{elements of list 1 <= dv}
      int64_t lo = 0, hi = n1;
      while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (d[off + mid] <= dv) lo = mid + 1; else hi = mid; }
      rank = u + lo;
    }
    ds[off + rank] = dv;
    zs[off + rank] = zv;
    perm[off + rank] = (int)t;
    dmax = fmax(dmax, fabs(dv));
  }
  // block max
  red[threadIdx.x] = dmax;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double rho = 2.0 * fabs(beta);
    rho_out[blockIdx.x] = rho;
    tol_out[blockIdx.x] = 8.0 * kU * fmax(red[0], rho);
  }
}

// ---------------------------------------------------------------- merge: deflation
// Sequential scan (one thread per merge).  Outputs at [off, off+m):
//   kind[t] = 0 nondeflated / 1 deflated; nd list (ascending) in ndl[off..off+k);
//   deflated list in dfl[off .. off+m-k); rotations (p, j, c, s) in rot arrays.
// Per merge: k, number of rotations.
// The merged block's columns are zero outside their half (Q1 rows 0..n1-1, Q2 rows
// n1..m-1) unless a deflation rotation mixed the two halves.  Each nondeflated
// column i gets a group (1: top rows only, 3: both, 2: bottom rows only) and its
// position pos[off+i] in the order [top | both | bottom] (ascending within a
// group), with grp[2 t] = #top, grp[2 t + 1] = #both: the product Qn U then splits
// into a top and a bottom product over column ranges of that order.
__global__ void k_dc_deflate(const MergeDesc* md, int count, double* ds, double* zs, const double* rho_in,
                             const double* tol_in, const int* perm, int* ndl, int* dfl, int* rotp, int* rotj,
                             double* rotc, double* rots, int* kout, int* nrot_out, int* pos, int* grp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const MergeDesc M = md[t];
  const int64_t off = M.off, m = M.n1 + M.n2;
  const double rho = rho_in[t], tol = tol_in[t];
  int k = 0, nd_df = 0, nr = 0;
  int pj = -1, ptype = 0;
  for (int j = 0; j < m; ++j) {
    if (rho * fabs(zs[off + j]) <= tol) { dfl[off + nd_df++] = j; continue; }
    const int bj = (perm[off + j] < M.n1) ? 1 : 2;
    if (pj < 0) { pj = j; ptype = bj; continue; }
    double s = zs[off + pj], c = zs[off + j];
    double r = hypot(s, c);
    double cc = c / r, ss = s / r;
    double tdiff = ds[off + j] - ds[off + pj];
    if (fabs(tdiff * cc * ss) <= tol) {
      zs[off + j] = r;
      zs[off + pj] = 0.0;
      double dp = ds[off + pj], dj = ds[off + j];
      ds[off + pj] = cc * cc * dp + ss * ss * dj;
      ds[off + j] = ss * ss * dp + cc * cc * dj;
      rotp[off + nr] = pj; rotj[off + nr] = j; rotc[off + nr] = cc; rots[off + nr] = ss; ++nr;
      dfl[off + nd_df++] = pj;
      pj = j;
      ptype |= bj;  // column j now holds a combination of both
    } else {
      pos[off + k] = ptype;
      ndl[off + k++] = pj;
      pj = j;
      ptype = bj;
    }
  }
  if (pj >= 0) {
    pos[off + k] = ptype;
    ndl[off + k++] = pj;
  }
  int c1 = 0, c2 = 0;
  for (int i = 0; i < k; ++i) {
    c1 += (pos[off + i] == 1);
    c2 += (pos[off + i] == 3);
  }
  int a1 = 0, a2 = c1, a3 = c1 + c2;
  for (int i = 0; i < k; ++i) {
    const int g = pos[off + i];
    pos[off + i] = (g == 1) ? a1++ : (g == 3) ? a2++ : a3++;
  }
  grp[2 * t] = c1;
  grp[2 * t + 1] = c2;
  kout[t] = k;
  nrot_out[t] = nr;
}

// Gather the block's columns in sorted order: Qt(:, t) = Qblock(:, perm[t]).
__global__ void k_dc_gather(const MergeDesc* md, const int* perm, const double* Q, int64_t ldq, double* Qt,
                            int64_t ldt) {
  const MergeDesc M = md[blockIdx.z];
  const int64_t off = M.off, m = M.n1 + M.n2;
  int64_t col = blockIdx.y;
  if (col >= m) return;
  int64_t src = perm[off + col];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
    Qt[(off + r) + (off + col) * ldt] = Q[(off + r) + (off + src) * ldq];
}

// Apply the deflation rotations in order, one thread per row.
__global__ void k_dc_rotate(const MergeDesc* md, const int* nrot, const int* rotp, const int* rotj,
                            const double* rotc, const double* rots, double* Qt, int64_t ldt) {
  const MergeDesc M = md[blockIdx.y];
  const int64_t off = M.off, m = M.n1 + M.n2;
  const int nr = nrot[blockIdx.y];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double* row = Qt + (off + r) + off * ldt;
    for (int q = 0; q < nr; ++q) {
      int64_t p = rotp[off + q], j = rotj[off + q];
      double c = rotc[off + q], s = rots[off + q];
      double qp = row[p * ldt], qj = row[j * ldt];
      row[p * ldt] = c * qp - s * qj;
      row[j * ldt] = s * qp + c * qj;
    }
  }
}

// Gather the nondeflated poles and z: dl[i] = ds[ndl[i]], zl[i] = zs[ndl[i]],
// and the nondeflated columns Qn(:, pos[i]) = Qt(:, ndl[i]) (grouped order).
__global__ void k_dc_gather_nd(const MergeDesc* md, const int* kk, const int* ndl, const int* pos, const double* ds,
                               const double* zs, double* dl, double* zl, const double* Qt, int64_t ldt, double* Qn) {
  const MergeDesc M = md[blockIdx.z];
  const int64_t off = M.off, m = M.n1 + M.n2;
  const int k = kk[blockIdx.z];
  int64_t i = blockIdx.y;
  if (i >= k) return;
  int64_t src = ndl[off + i];
  if (blockIdx.x == 0 && threadIdx.x == 0) { dl[off + i] = ds[off + src]; zl[off + i] = zs[off + src]; }
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
    Qn[(off + r) + (off + pos[off + i]) * ldt] = Qt[(off + r) + (off + src) * ldt];
}

// ---------------------------------------------------------------- secular equation
// Root i of 1 + rho sum_j z_j^2 / (d_j - lambda) = 0, poles d (ascending, k of them).
// lambda_i = d[org_i] + tau_i.  Bracketed middle-way iteration with bisection fallback.
__device__ void secular_root(int i, int k, const double* dl, const double* zl, double rho, int* org_out,
                             double* tau_out, int* st, int info) {
  if (k == 1) { *org_out = 0; *tau_out = rho * zl[0] * zl[0]; return; }
  int org;
  double lo, hi, tau;
  if (i < k - 1) {
    const double gap = dl[i + 1] - dl[i];
    const double mid = 0.5 * gap;
    double f = 1.0;
    for (int j = 0; j < k; ++j) f += rho * zl[j] * zl[j] / ((dl[j] - dl[i]) - mid);
    if (f >= 0.0) { org = i; lo = 0.0; hi = mid; }
    else { org = i + 1; lo = -mid; hi = 0.0; }
    tau = 0.5 * (lo + hi);
  } else {
    org = k - 1;
    double zz = 0.0;
    for (int j = 0; j < k; ++j) zz += zl[j] * zl[j];
    lo = 0.0; hi = rho * zz;
    tau = 0.5 * hi;
  }
  const double dorg = dl[org];
  bool conv = false;
  for (int it = 0; it < 120; ++it) {
    double psi = 0.0, dpsi = 0.0, phi = 0.0, dphi = 0.0;
    // one reciprocal per pole (FP64 division is the costly operation here): the
    // term rho z_j^2 / del and its derivative rho z_j^2 / del^2 share it
    for (int j = 0; j <= i; ++j) {
      const double r = 1.0 / ((dl[j] - dorg) - tau);
      const double t = (rho * zl[j] * zl[j]) * r;
      psi += t;
      dpsi = fma(t, r, dpsi);
    }
    for (int j = i + 1; j < k; ++j) {
      const double r = 1.0 / ((dl[j] - dorg) - tau);
      const double t = (rho * zl[j] * zl[j]) * r;
      phi += t;
      dphi = fma(t, r, dphi);
    }
    const double g = 1.0 + psi + phi;
    const double erretm = 1.0 + fabs(psi) + fabs(phi);
    if (fabs(g) <= 16.0 * kU * erretm * (double)(k < 8 ? 8 : k) / 8.0) { conv = true; break; }
    if (g > 0.0) hi = tau; else lo = tau;
    // the bracket is tight relative to tau itself (tau is the distance to the pole,
    // which the eigenvector formula divides by)
    if (!(hi - lo > 2.0 * kU * fmax(fabs(lo), fabs(hi)))) { conv = true; break; }
    double eta;
    const double Di = (dl[i] - dorg) - tau;
    if (i < k - 1) {
      const double Dn = (dl[i + 1] - dorg) - tau;
      const double c = g - Di * dpsi - Dn * dphi;
      const double s = Di * Di * dpsi, S = Dn * Dn * dphi;
      const double A = c, B = -(c * (Di + Dn) + s + S), C = c * Di * Dn + s * Dn + S * Di;
      double r1, r2;
      if (fabs(A) <= 1e-300 * (fabs(B) + fabs(C))) {
        r1 = r2 = (B != 0.0) ? -C / B : 0.5 * (lo + hi) - tau;
      } else {
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) disc = 0.0;
        double q = -0.5 * (B + copysign(sqrt(disc), B));
        r1 = q / A;
        r2 = (q != 0.0) ? C / q : r1;
      }
      double t1 = tau + r1, t2 = tau + r2;
      bool in1 = (t1 > lo && t1 < hi), in2 = (t2 > lo && t2 < hi);
      if (in1 && in2) eta = (fabs(r1) < fabs(r2)) ? r1 : r2;
      else if (in1) eta = r1;
      else if (in2) eta = r2;
      else eta = 0.5 * (lo + hi) - tau;
    } else {
      const double c = g - Di * dpsi;
      const double s = Di * Di * dpsi;
      eta = (c != 0.0) ? Di + s / c : 0.5 * (lo + hi) - tau;
      double t1 = tau + eta;
      if (!(t1 > lo && t1 < hi)) eta = 0.5 * (lo + hi) - tau;
    }
    double nt = tau + eta;
    if (!(nt > lo && nt < hi) || !isfinite(nt)) nt = 0.5 * (lo + hi);
    tau = nt;
  }
  if (!conv) dev_set_status(st, EVD_ERR_NO_CONVERGENCE, info);
  *org_out = org;
  *tau_out = tau;
}

__global__ void k_dc_secular(const MergeDesc* md, const int* kk, const double* dl, const double* zl,
                             const double* rho_in, int* org, double* tau, int* st) {
  const MergeDesc M = md[blockIdx.y];
  const int k = kk[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const int64_t off = M.off;
  int o;
  double t;
  secular_root(i, k, dl + off, zl + off, rho_in[blockIdx.y], &o, &t, st, (int)(off + i + 1));
  org[off + i] = o;
  tau[off + i] = t;
}

// Loewner formula: zhat_j^2 = prod_i (lambda_i - d_j) / (rho prod_{i != j} (d_i - d_j)).
__global__ void k_dc_lowner(const MergeDesc* md, const int* kk, const double* dl, const double* zl,
                            const double* rho_in, const int* org, const double* tau, double* zh) {
  const MergeDesc M = md[blockIdx.y];
  const int k = kk[blockIdx.y];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int64_t off = M.off;
  const double rho = rho_in[blockIdx.y];
  const double dj = dl[off + j];
  // the products of the numerators and of the denominators are kept apart, each
  // rescaled to [0.5, 1) every 8 factors with its binary exponent counted, so the
  // k - 1 factors cost multiplications and one division at the end
  double num = ((dl[off + org[off + j]] - dj) + tau[off + j]) / rho, den = 1.0;
  int enum_ = 0, eden = 0;
  int cnt = 0;
  for (int i = 0; i < k; ++i) {
    if (i == j) continue;
    num *= (dl[off + org[off + i]] - dj) + tau[off + i];
    den *= dl[off + i] - dj;
    if (++cnt == 8) {
      int e1, e2;
      num = frexp(num, &e1);
      den = frexp(den, &e2);
      enum_ += e1;
      eden += e2;
      cnt = 0;
    }
  }
  const double w = ldexp(num / den, enum_ - eden);
  zh[off + j] = copysign(sqrt(fabs(w)), zl[off + j]);
}

// Eigenvector i of D + rho zhat zhat^T: u(j) = zhat_j / (d_j - lambda_i), normalised.
// Written as column i of the k x k matrix U at the merge's diagonal block (ld ldu).
// Column i of U (root i), its rows in the grouped order of the poles (pos).
__global__ void k_dc_vectors(const MergeDesc* md, const int* kk, const double* dl, const int* org,
                             const double* tau, const double* zh, const int* pos, double* U, int64_t ldu) {
  const MergeDesc M = md[blockIdx.y];
  const int k = kk[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const int64_t off = M.off;
  const double dorg = dl[off + org[off + i]], ti = tau[off + i];
  double ss = 0.0;
  for (int j = 0; j < k; ++j) {
    double u = zh[off + j] / ((dl[off + j] - dorg) - ti);
    ss += u * u;
  }
  const double inv = 1.0 / sqrt(ss);
  double* col = U + off + (off + i) * ldu;
  for (int j = 0; j < k; ++j) col[pos[off + j]] = zh[off + j] / ((dl[off + j] - dorg) - ti) * inv;
}

__device__ __forceinline__ long long order_key(double x) {
  long long b = __double_as_longlong(x);
  return (b < 0) ? (long long)(0x8000000000000000ull - (unsigned long long)b) - 1 : b + 0;
}

// Final order of the merged eigenpairs: values lambda_i (nondeflated, in order)
// and the deflated poles; rank by counting (ties by source index).  Then gather
// the eigenvector columns: lambda columns from X (the product Qn U, stored in the
// block's first k columns of Q) and deflated columns from Qt.  Destination: Qn.
__global__ void k_dc_rank(const MergeDesc* md, const int* kk, const double* dl, const int* org, const double* tau,
                          const double* ds, const int* dfl, double* vals, int* rank) {
  const MergeDesc M = md[blockIdx.y];
  const int64_t off = M.off, m = M.n1 + M.n2;
  const int k = kk[blockIdx.y];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  // value of item t: t < k -> lambda_t, else deflated pole dfl[t-k]
  auto val = [&](int64_t q) -> double {
    if (q < k) return dl[off + org[off + q]] + tau[off + q];
    return ds[off + dfl[off + (q - k)]];
  };
  const double v = val(t);
  const long long key = order_key(v);
  int64_t r = 0;
  for (int64_t q = 0; q < m; ++q) {
    long long kq = order_key(val(q));
    if (kq < key || (kq == key && q < t)) ++r;
  }
  vals[off + r] = v;
  rank[off + t] = (int)r;
}

__global__ void k_dc_assemble(const MergeDesc* md, const int* kk, const int* rank, const int* dfl, const double* Q,
                              int64_t ldq, const double* Qt, int64_t ldt, double* Qdst) {
  const MergeDesc M = md[blockIdx.z];
  const int64_t off = M.off, m = M.n1 + M.n2;
  const int k = kk[blockIdx.z];
  const int64_t t = blockIdx.y;
  if (t >= m) return;
  const int64_t dst = rank[off + t];
  const double* src = (t < k) ? Q + off + (off + t) * ldq : Qt + off + (off + dfl[off + (t - k)]) * ldt;
  const int64_t lds = 1;
  (void)lds;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
    Qdst[(off + r) + (off + dst) * ldt] = src[r];
}

__global__ void k_dc_copy_back(const MergeDesc* md, const double* vals, double* d, const double* Qs, int64_t lds,
                               double* Q, int64_t ldq) {
  const MergeDesc M = md[blockIdx.z];
  const int64_t off = M.off, m = M.n1 + M.n2;
  const int64_t c = blockIdx.y;
  if (c >= m) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) d[off + c] = vals[off + c];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
    Q[(off + r) + (off + c) * ldq] = Qs[(off + r) + (off + c) * lds];
}

// Sync-free merges (no host read of k): the product runs over the whole merge, so
// the columns of Qn past the k nondeflated ones and U past its k x k block must be
// zero (stale values there, even non-finite ones, would otherwise reach the first k
// columns of the product).
__global__ void k_dc_pad_zero(const MergeDesc* md, const int* kk, double* Qn, double* U, int64_t ld) {
  const MergeDesc M = md[blockIdx.z];
  const int64_t off = M.off, m = M.n1 + M.n2;
  const int k = kk[blockIdx.z];
  const int64_t c = blockIdx.y;
  if (c >= m) return;
  double* qc = Qn + off + (off + c) * ld;
  double* uc = U + off + (off + c) * ld;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    if (c >= k) {
      qc[r] = 0.0;
      uc[r] = 0.0;
    } else if (r >= k) {
      uc[r] = 0.0;
    }
  }
}

__global__ void k_zero_cols(double* Q, int64_t ldq, int64_t n, int64_t j0) {
  int64_t j = j0 + blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Q[i + j * ldq] = 0.0;
}

void build_tree(int64_t off, int64_t n, int depth, std::vector<std::vector<MergeDesc>>& levels,
                std::vector<int64_t>& loff, std::vector<int>& ln) {
  if (n <= LEAF) { loff.push_back(off); ln.push_back((int)n); return; }
  int64_t n1 = n / 2, n2 = n - n1;
  build_tree(off, n1, depth + 1, levels, loff, ln);
  build_tree(off + n1, n2, depth + 1, levels, loff, ln);
  if ((int)levels.size() <= depth) levels.resize(depth + 1);
  levels[depth].push_back({off, n1, n2});
}

}  // namespace

// The merge tree of order n: descriptors level by level, deepest first (the order
// dc_run walks them), and the leaves.  It depends on n only.
void dc_tree(int64_t n, std::vector<MergeDesc>& all, std::vector<size_t>& lvl_start, std::vector<int64_t>& loff,
             std::vector<int>& ln) {
  std::vector<std::vector<MergeDesc>> levels;
  build_tree(0, n, 0, levels, loff, ln);
  for (int L = (int)levels.size() - 1; L >= 0; --L) {
    lvl_start.push_back(all.size());
    for (auto& m : levels[L]) all.push_back(m);
  }
  lvl_start.push_back(all.size());
}


size_t dc_tree_bytes(int64_t n) {
  if (n <= 0) return 256;
  std::vector<MergeDesc> all;
  std::vector<size_t> lvl;
  std::vector<int64_t> loff;
  std::vector<int> ln;
  dc_tree(n, all, lvl, loff, ln);
  return align_up(sizeof(MergeDesc) * (all.size() + 1), 256) + align_up(sizeof(int64_t) * loff.size(), 256) +
         align_up(sizeof(int) * ln.size(), 256);
}

evd_status_t dc_tree_upload(int64_t n, void* dst, size_t bytes) {
  if (n <= 0) return EVD_OK;
  std::vector<MergeDesc> all;
  std::vector<size_t> lvl;
  std::vector<int64_t> loff;
  std::vector<int> ln;
  dc_tree(n, all, lvl, loff, ln);
  if (bytes < dc_tree_bytes(n)) return EVD_ERR_INVALID_ARG;
  char* p = static_cast<char*>(dst);
  const size_t a = align_up(sizeof(MergeDesc) * (all.size() + 1), 256), b = align_up(sizeof(int64_t) * loff.size(), 256);
  if (!all.empty()) EVD_CUDA_TRY(cudaMemcpy(p, all.data(), sizeof(MergeDesc) * all.size(), cudaMemcpyHostToDevice));
  EVD_CUDA_TRY(cudaMemcpy(p + a, loff.data(), sizeof(int64_t) * loff.size(), cudaMemcpyHostToDevice));
  EVD_CUDA_TRY(cudaMemcpy(p + a + b, ln.data(), sizeof(int) * ln.size(), cudaMemcpyHostToDevice));
  return EVD_OK;
}


evd_status_t dc_run(const PlanCore& pc, double* d, double* e, double* Q, int64_t ldq, const DcWork& w) {
  const int64_t n = pc.n;
  cudaStream_t s = pc.stream;
  if (n == 0) return EVD_OK;
  std::vector<MergeDesc> all;
  std::vector<size_t> lvl_start;
  std::vector<int64_t> loff;
  std::vector<int> ln;
  dc_tree(n, all, lvl_start, loff, ln);
  // vector scratch (DcWork::vec holds 10 n doubles, DcWork::ivec 32 n ints)
  double* ds = w.vec;
  double* zs = w.vec + n;
  double* dl = w.vec + 2 * n;
  double* zl = w.vec + 3 * n;
  double* tau = w.vec + 4 * n;
  double* zh = w.vec + 5 * n;
  double* vals = w.vec + 6 * n;
  double* rotc = w.vec + 7 * n;
  double* rots = w.vec + 8 * n;
  int* perm = w.ivec;
  int* ndl = w.ivec + n;
  int* dfl = w.ivec + 2 * n;
  int* rotp = w.ivec + 3 * n;
  int* rotj = w.ivec + 4 * n;
  int* org = w.ivec + 5 * n;
  int* rank = w.ivec + 6 * n;
  int* pos = w.ivec + 7 * n;
  // merge descriptors and per-merge scalars
  const size_t nmerge = all.size(), nleaves = loff.size();
  char* meta = reinterpret_cast<char*>(w.ivec + 8 * n);
  size_t mb = 0;
  auto carve = [&](size_t bytes) { char* p = meta + mb; mb += align_up(bytes, 256); return p; };
  MergeDesc* d_md = reinterpret_cast<MergeDesc*>(carve(sizeof(MergeDesc) * (nmerge + 1)));
  int64_t* d_loff = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * nleaves));
  int* d_ln = reinterpret_cast<int*>(carve(sizeof(int) * nleaves));
  double* d_rho = reinterpret_cast<double*>(carve(sizeof(double) * (nmerge + 1)));
  double* d_tol = reinterpret_cast<double*>(carve(sizeof(double) * (nmerge + 1)));
  int* d_k = reinterpret_cast<int*>(carve(sizeof(int) * (nmerge + 1)));
  int* d_nrot = reinterpret_cast<int*>(carve(sizeof(int) * (nmerge + 1)));
  int* d_grp = reinterpret_cast<int*>(carve(sizeof(int) * 2 * (nmerge + 1)));
  // descriptors of one level's small merge products (two per merge), launched together
  Gemm* d_gd = reinterpret_cast<Gemm*>(carve(sizeof(Gemm) * 2 * (nmerge + 1)));
  std::vector<Gemm> small_gd;
  if (mb > ((size_t)24 * n + 1024) * sizeof(int)) return ws_fail("dc merge descriptors", ((size_t)24 * n + 1024) * sizeof(int), mb);
  if (pc.dc_tree) {
    // the plan's resident copy of the tree (uploaded once, at plan creation)
    char* t = static_cast<char*>(pc.dc_tree);
    d_md = reinterpret_cast<MergeDesc*>(t);
    d_loff = reinterpret_cast<int64_t*>(t + align_up(sizeof(MergeDesc) * (nmerge + 1), 256));
    d_ln = reinterpret_cast<int*>(t + align_up(sizeof(MergeDesc) * (nmerge + 1), 256) +
                                  align_up(sizeof(int64_t) * nleaves, 256));
  } else {
    if (pc.dc_sync_free) return EVD_ERR_INVALID_ARG;  // a captured solve cannot copy from transient host memory
    if (nmerge) EVD_CUDA_TRY(cudaMemcpyAsync(d_md, all.data(), sizeof(MergeDesc) * nmerge, cudaMemcpyHostToDevice, s));
    EVD_CUDA_TRY(cudaMemcpyAsync(d_loff, loff.data(), sizeof(int64_t) * nleaves, cudaMemcpyHostToDevice, s));
    EVD_CUDA_TRY(cudaMemcpyAsync(d_ln, ln.data(), sizeof(int) * nleaves, cudaMemcpyHostToDevice, s));
  }
  // Q = 0, tears, leaves
  for (int64_t j0 = 0; j0 < n; j0 += 65535) {
    int64_t cols = n - j0 < 65535 ? n - j0 : 65535;
    k_zero_cols<<<dim3(4, (unsigned)cols), 256, 0, s>>>(Q, ldq, n, j0); count_launch();
  }
  if (nmerge) k_dc_tear<<<(unsigned)ceil_div(nmerge, 128), 128, 0, s>>>(d_md, (int)nmerge, d, e); count_launch();
  {
    StatScope sc_leaf("dc_leaf", s);
    k_dc_leaf<<<(unsigned)ceil_div(nleaves * 32, 128), 128, 0, s>>>(d_loff, d_ln, (int)nleaves, d, e, Q, ldq,
                                                                     pc.status); count_launch();
  }
  EVD_CUDA_TRY(cudaGetLastError());
  std::vector<int> hk(nmerge + 1), hg(2 * (nmerge + 1));
  for (size_t L = 0; L + 1 < lvl_start.size(); ++L) {
    const size_t b0 = lvl_start[L], cnt = lvl_start[L + 1] - b0;
    if (cnt == 0) continue;
    MergeDesc* md = d_md + b0;
    int64_t mmax = 0;
    for (size_t q = 0; q < cnt; ++q) mmax = std::max<int64_t>(mmax, all[b0 + q].n1 + all[b0 + q].n2);
    const unsigned rx = (unsigned)std::min<int64_t>(ceil_div(mmax, 256), 8);
    { StatScope sc("dc_merge", s);
    k_dc_prepare<<<(unsigned)cnt, 256, 0, s>>>(md, d, e, Q, ldq, ds, zs, perm, d_rho + b0, d_tol + b0); count_launch();
    k_dc_deflate<<<(unsigned)ceil_div(cnt, 64), 64, 0, s>>>(md, (int)cnt, ds, zs, d_rho + b0, d_tol + b0, perm, ndl,
                                                            dfl, rotp, rotj, rotc, rots, d_k + b0, d_nrot + b0, pos,
                                                            d_grp + 2 * b0); count_launch();
    k_dc_gather<<<dim3(rx, (unsigned)mmax, (unsigned)cnt), 256, 0, s>>>(md, perm, Q, ldq, w.Qtmp, n); count_launch();
    k_dc_rotate<<<dim3((unsigned)ceil_div(mmax, 128), (unsigned)cnt), 128, 0, s>>>(md, d_nrot + b0, rotp, rotj, rotc,
                                                                                 rots, w.Qtmp, n); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
    }
    // the number of nondeflated roots sizes the products: read it on the host, or,
    // sync-free, size every grid and product by the merge itself
    int kmax = 0;
    if (pc.dc_sync_free) {
      kmax = (int)mmax;
    } else {
      EVD_CUDA_TRY(cudaMemcpyAsync(hk.data(), d_k + b0, sizeof(int) * cnt, cudaMemcpyDeviceToHost, s));
      EVD_CUDA_TRY(cudaMemcpyAsync(hg.data(), d_grp + 2 * b0, sizeof(int) * 2 * cnt, cudaMemcpyDeviceToHost, s));
      EVD_CUDA_TRY(cudaStreamSynchronize(s));
      for (size_t q = 0; q < cnt; ++q) kmax = std::max(kmax, hk[q]);
    }
    if (kmax > 0) {
      k_dc_gather_nd<<<dim3(rx, (unsigned)kmax, (unsigned)cnt), 256, 0, s>>>(md, d_k + b0, ndl, pos, ds, zs, dl, zl,
                                                                             w.Qtmp, n, w.Qn); count_launch();
      const unsigned kx = (unsigned)ceil_div(kmax, 128);
      { StatScope sc("dc_secular", s);
      k_dc_secular<<<dim3(kx, (unsigned)cnt), 128, 0, s>>>(md, d_k + b0, dl, zl, d_rho + b0, org, tau, pc.status); count_launch();
      k_dc_lowner<<<dim3(kx, (unsigned)cnt), 128, 0, s>>>(md, d_k + b0, dl, zl, d_rho + b0, org, tau, zh); count_launch();
      k_dc_vectors<<<dim3(kx, (unsigned)cnt), 128, 0, s>>>(md, d_k + b0, dl, org, tau, zh, pos, w.Umat, n); count_launch();
      EVD_CUDA_TRY(cudaGetLastError());
      }
      if (pc.dc_sync_free) {
        // X = Qn U over the whole merge block, Qn and U zero past the k nondeflated
        // columns (and rows of U); X's columns from k on are not read
        k_dc_pad_zero<<<dim3(rx, (unsigned)mmax, (unsigned)cnt), 256, 0, s>>>(md, d_k + b0, w.Qn, w.Umat, n); count_launch();
        EVD_CUDA_TRY(cudaGetLastError());
        for (size_t q = 0; q < cnt; ++q) {
          const MergeDesc& M = all[b0 + q];
          const int64_t off = M.off, m = M.n1 + M.n2;
          Gemm g;
          g.tag = "dc_merge_gemm";
          g.status = pc.status;
          g.m = m; g.n = m; g.k = m;
          g.A = w.Qn + off + off * n; g.lda = n;
          g.B = w.Umat + off + off * n; g.ldb = n;
          g.C = Q + off + off * ldq; g.ldc = ldq;
          g.alpha = 1.0; g.beta = 0.0;
          evd_status_t st = gemm(g, pc.ref_slices, w.gemm_ws, w.gemm_ws_bytes, s);
          if (st != EVD_OK) return st;
        }
      }
      // X = Qn U into the first k columns of the block of Q (the block is free now),
      // as X(0:n1, :) = Qn(0:n1, 0:c1+c2) U(0:c1+c2, :) and
      //    X(n1:m, :) = Qn(n1:m, c1:k)     U(c1:k, :)
      small_gd.clear();
      for (size_t q = 0; q < cnt && !pc.dc_sync_free; ++q) {
        const int k = hk[q];
        if (k == 0) continue;
        const MergeDesc& M = all[b0 + q];
        const int64_t off = M.off, n1 = M.n1, n2 = M.n2;
        const int c1 = hg[2 * q], c2 = hg[2 * q + 1];
        for (int half = 0; half < 2; ++half) {
          const int64_t r0 = half ? n1 : 0, rows = half ? n2 : n1;
          const int64_t j0 = half ? c1 : 0, kk = half ? (int64_t)k - c1 : (int64_t)c1 + c2;
          Gemm g;
          g.tag = "dc_merge_gemm";
          g.status = pc.status;
          g.m = rows; g.n = k; g.k = kk;
          g.A = w.Qn + (off + r0) + (off + j0) * n; g.lda = n;
          g.B = w.Umat + (off + j0) + off * n; g.ldb = n;
          g.C = Q + (off + r0) + off * ldq; g.ldc = ldq;
          g.alpha = 1.0; g.beta = 0.0;
          if (g.m <= 0 || g.n <= 0 || g.k <= 0) continue;
          if (!ozaki_eligible(g)) {
            small_gd.push_back(g);  // FP64 CUDA cores, with the level's other small products
            continue;
          }
          // FP64-accurate in every mode: the next merge's z is the last row of Q1 and the
          // first of Q2, and a product error at the slice level would blur the tiny
          // entries that deflate
          evd_status_t st = gemm(g, pc.ref_slices, w.gemm_ws, w.gemm_ws_bytes, s);
          if (st != EVD_OK) return st;
        }
      }
      {
        const evd_status_t st = gemm_simt_batched(small_gd.data(), (int)small_gd.size(), d_gd, "dc_merge_gemm", s);
        if (st != EVD_OK) return st;
      }
    }
    StatScope sc2("dc_merge", s);
    k_dc_rank<<<dim3((unsigned)ceil_div(mmax, 128), (unsigned)cnt), 128, 0, s>>>(md, d_k + b0, dl, org, tau, ds, dfl,
                                                                               vals, rank); count_launch();
    k_dc_assemble<<<dim3(rx, (unsigned)mmax, (unsigned)cnt), 256, 0, s>>>(md, d_k + b0, rank, dfl, Q, ldq, w.Qtmp, n,
                                                                          w.Qn); count_launch();
    k_dc_copy_back<<<dim3(rx, (unsigned)mmax, (unsigned)cnt), 256, 0, s>>>(md, vals, d, w.Qn, n, Q, ldq); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
  }
  return EVD_OK;
}

}  // namespace evd
