// Bulge chasing: band (half-width b) -> symmetric tridiagonal (Sec. 2.1.1, Sec. 4.2).
//
// Sweep j (j = 0 .. n-3) reduces column j.  Step k works on the rows
// R_k = [r0, r1], r0 = j + 1 + k b, r1 = min(r0 + b - 1, n - 1):
//   * the reflector H = I - tau v v^T (v0 = 1, LAPACK sign choice) annihilates
//     A(r0+1 : r1, c) with c = j for k = 0 and c = r0 - b (the first column of the
//     bulge the previous step created) for k >= 1;
//   * H is applied from the left to the rest of that bulge, A(R_k, c+1 : r0-1),
//     two-sided to the diagonal block A(R_k, R_k), and from the right to the block
//     below, A(r1+1 : r1+b, R_k), which creates the next bulge.
// The band lives in (2b+1) x n lower band storage (room for the bulge) in global
// memory, which for the sizes of interest stays in the 129 MB L2.
//
// Concurrency (the single-GPU form of the pipelined BC): one cooperative launch,
// CTA g runs sweeps j = g, g + G, ...  Before step k of sweep j it waits (bounded)
// until sweep j-1 has completed step k+2: the rows and columns step k of sweep j
// touches are [r0, r1 + b] x [r0 - b, r1], so step k of sweep j and step k' >= k+3
// of sweep j-1 touch disjoint entries, and every entry sweep j reads has already
// received all of sweep j-1's updates that precede it in sweep order.
#include <climits>
#include <cstdlib>
#include <cstdio>

#include "device_util.cuh"
#include "evd_internal.h"

namespace evd {

namespace {

constexpr int BC_NT = 128;
constexpr int BC_LAG = 3;  // sweep j step k waits for sweep j-1 to finish step k + BC_LAG - 1
constexpr int BC_LAG_CARRY = 2;  // the look-ahead form publishes beta one step early

// Number of steps of sweep j: steps with |R_k| >= 2.
__host__ __device__ inline int64_t sweep_steps(int64_t n, int b, int64_t j) {
  if (j + 3 > n) return 0;
  return (n - 3 - j) / b + 1;
}
// F(T) = sum_{t=0}^{T} floor(t / b)
__host__ __device__ inline int64_t floor_sum(int64_t T, int b) {
  if (T < 0) return 0;
  int64_t q = T / b;
  return (int64_t)b * q * (q - 1) / 2 + q * (T - q * b + 1);
}
// Index of the first reflector of sweep j (sweeps stored one after another).
__host__ __device__ inline int64_t sweep_offset(int64_t n, int b, int64_t j) {
  int64_t jj = j < n - 2 ? j : (n - 2 > 0 ? n - 2 : 0);
  if (n < 3) return 0;
  return floor_sum(n - 3, b) - floor_sum(n - 3 - jj, b) + jj;
}

struct BcArgs {
  double* band;
  int64_t n;
  int b;
  double* U;      // nullptr when vectors are not wanted
  double* Utau;
  int* prog;
  int* st;
};

// Band entries are read and written through L2 only (ld.cg / st.cg): other CTAs
// (other sweeps) update them, and L1 is not coherent across SMs.
__device__ __forceinline__ double bget(const double* band, int ldb, int64_t r, int64_t c) {
  return __ldcg(band + (r - c) + c * ldb);
}
__device__ __forceinline__ void bput(double* band, int ldb, int64_t r, int64_t c, double x) {
  __stcg(band + (r - c) + c * ldb, x);
}

__global__ void __launch_bounds__(BC_NT) k_bulge_chase(const BcArgs a) {
  __shared__ double v[128];
  __shared__ double wv[128];
  __shared__ double red[BC_NT];
  __shared__ double par[4];
  const int b = a.b, ldb = 2 * b + 1;
  const int64_t n = a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = BC_NT / 32;
  for (int64_t j = blockIdx.x; j + 3 <= n; j += gridDim.x) {
    const int64_t K = sweep_steps(n, b, j);
    const int64_t Kprev = (j > 0) ? sweep_steps(n, b, j - 1) : 0;
    const int64_t uoff = sweep_offset(n, b, j);
    for (int64_t k = 0; k < K; ++k) {
      if (j > 0) {
        int64_t need = k + BC_LAG;
        if (need > Kprev) need = Kprev;
        if (threadIdx.x == 0) {
          if (!wait_geq(a.prog + (j - 1), (int)need, a.st, (int)(j + 1))) par[3] = 1.0; else par[3] = 0.0;
        }
        __syncthreads();
        if (par[3] != 0.0) return;
      }
      const int64_t r0 = j + 1 + k * b;
      const int64_t r1 = (r0 + b - 1 < n - 1) ? r0 + b - 1 : n - 1;
      const int m = (int)(r1 - r0 + 1);
      const int64_t c = (k == 0) ? j : r0 - b;
      // ---- reflector from x = A(R_k, c)
      double x = 0.0;
      if (threadIdx.x < m) x = bget(a.band, ldb, r0 + threadIdx.x, c);
      double ss = (threadIdx.x >= 1 && threadIdx.x < m) ? x * x : 0.0;
      ss = block_sum<BC_NT>(ss, red);
      if (threadIdx.x == 0) {
        double alpha = x, tau = 0.0, beta = alpha, scale = 0.0;
        if (ss != 0.0) {
          double nrm = sqrt(alpha * alpha + ss);
          beta = (alpha >= 0.0) ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        par[0] = tau; par[1] = beta; par[2] = scale;
      }
      __syncthreads();
      const double tau = par[0], beta = par[1], scale = par[2];
      if (threadIdx.x < b) v[threadIdx.x] = (threadIdx.x == 0) ? 1.0 : (threadIdx.x < m ? x * scale : 0.0);
      __syncthreads();
      if (a.U) {
        const int64_t idx = uoff + k;
        if (threadIdx.x < b) a.U[idx * b + threadIdx.x] = v[threadIdx.x];
        if (threadIdx.x == 0) a.Utau[idx] = tau;
      }
      // annihilated column
      if (threadIdx.x < m) bput(a.band, ldb, r0 + threadIdx.x, c, (threadIdx.x == 0) ? beta : 0.0);
      if (tau != 0.0) {
        // ---- left application to the rest of the bulge: columns c+1 .. r0-1 (k >= 1)
        for (int64_t cc = c + 1 + warp; cc < r0; cc += nwarps) {
          double s = 0.0;
          for (int t = lane; t < m; t += 32) s += v[t] * bget(a.band, ldb, r0 + t, cc);
          s = warp_sum(s) * tau;
          for (int t = lane; t < m; t += 32) bput(a.band, ldb, r0 + t, cc, bget(a.band, ldb, r0 + t, cc) - s * v[t]);
        }
        // ---- two-sided on the diagonal block D = A(R_k, R_k)
        for (int p = threadIdx.x; p < m; p += BC_NT) {
          double s = 0.0;
          for (int q = 0; q < m; ++q) {
            double dpq = (p >= q) ? bget(a.band, ldb, r0 + p, r0 + q) : bget(a.band, ldb, r0 + q, r0 + p);
            s += dpq * v[q];
          }
          wv[p] = tau * s;
        }
        __syncthreads();
        double pv = (threadIdx.x < m) ? wv[threadIdx.x] * v[threadIdx.x] : 0.0;
        pv = block_sum<BC_NT>(pv, red);
        const double alpha = 0.5 * tau * pv;
        if (threadIdx.x < m) wv[threadIdx.x] -= alpha * v[threadIdx.x];
        __syncthreads();
        for (int idx = threadIdx.x; idx < m * m; idx += BC_NT) {
          int p = idx % m, q = idx / m;
          if (p >= q) bput(a.band, ldb, r0 + p, r0 + q, bget(a.band, ldb, r0 + p, r0 + q) - (v[p] * wv[q] + wv[p] * v[q]));
        }
        // ---- right application to the block below: rows r1+1 .. min(r1+b, n-1)
        const int64_t rb_end = (r1 + b < n - 1) ? r1 + b : n - 1;
        for (int64_t r = r1 + 1 + warp; r <= rb_end; r += nwarps) {
          double s = 0.0;
          for (int t = lane; t < m; t += 32) s += bget(a.band, ldb, r, r0 + t) * v[t];
          s = warp_sum(s) * tau;
          for (int t = lane; t < m; t += 32) bput(a.band, ldb, r, r0 + t, bget(a.band, ldb, r, r0 + t) - s * v[t]);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        st_release(a.prog + j, (int)(k + 1));
      }
    }
    if (K == 0 && threadIdx.x == 0) st_release(a.prog + j, 0);
  }
}

// Shared-memory-staged form of the same step (b <= BM): the three blocks a step
// touches -- the bulge A(R_k, c : r0-1), the diagonal block A(R_k, R_k) and the
// block below A(r1+1 : r1+b, R_k) -- are read from the band once with coalesced
// loads, updated in shared memory, and written back once.  Identical arithmetic to
// k_bulge_chase, in the same order per entry.
template <int BM>
__global__ void __launch_bounds__(BC_NT) k_bulge_chase_smem(const BcArgs a) {
  extern __shared__ double smb[];
  constexpr int LD = BM + 1;
  double* Ls = smb;             // Ls[t * LD + cc] = A(r0 + t, c + cc)
  double* Ds = Ls + BM * LD;    // Ds[q * LD + p]  = A(r0 + p, r0 + q)   (both triangles)
  double* Bs = Ds + BM * LD;    // Bs[t * LD + rr] = A(r1 + 1 + rr, r0 + t)
  __shared__ double v[BM], wv[BM];
  __shared__ double par[4];
  const int b = a.b, ldb = 2 * b + 1;
  const int64_t n = a.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t j = blockIdx.x; j + 3 <= n; j += gridDim.x) {
    const int64_t K = sweep_steps(n, b, j);
    const int64_t Kprev = (j > 0) ? sweep_steps(n, b, j - 1) : 0;
    const int64_t uoff = sweep_offset(n, b, j);
    for (int64_t k = 0; k < K; ++k) {
      if (j > 0) {
        int64_t need = k + BC_LAG;
        if (need > Kprev) need = Kprev;
        if (tid == 0) par[3] = wait_geq(a.prog + (j - 1), (int)need, a.st, (int)(j + 1)) ? 0.0 : 1.0;
        __syncthreads();
        if (par[3] != 0.0) return;
      }
      const int64_t r0 = j + 1 + k * b;
      const int64_t r1 = (r0 + b - 1 < n - 1) ? r0 + b - 1 : n - 1;
      const int m = (int)(r1 - r0 + 1);
      const int64_t c = (k == 0) ? j : r0 - b;
      const int ncol = (int)(r0 - c);                                   // 1 for k = 0, b otherwise
      const int mb = (int)(((r1 + b < n - 1) ? r1 + b : n - 1) - r1);   // rows of the block below
      // ---- load (2-D thread mapping: row = tid % BM, column stride BC_NT / BM)
      constexpr int CS = BC_NT / BM;
      const int tr = tid % BM, tc = tid / BM;
      if (tr < m) {
        for (int cc = tc; cc < ncol; cc += CS) Ls[tr * LD + cc] = bget(a.band, ldb, r0 + tr, c + cc);
        for (int q = tc; q <= tr; q += CS) Ds[q * LD + tr] = bget(a.band, ldb, r0 + tr, r0 + q);
      }
      if (tr < mb)
        for (int t = tc; t < m; t += CS) Bs[t * LD + tr] = bget(a.band, ldb, r1 + 1 + tr, r0 + t);
      __syncthreads();
      if (tr < m)
        for (int q = tc; q < m; q += CS)
          if (tr < q) Ds[q * LD + tr] = Ds[tr * LD + q];
      // ---- reflector from x = Ls(:, 0)
      if (warp == 0) {
        double ss = 0.0;
        for (int t = 1 + lane; t < m; t += 32) { const double x = Ls[t * LD]; ss += x * x; }
        ss = warp_sum(ss);
        if (lane == 0) {
          const double alpha = Ls[0];
          double tau = 0.0, beta = alpha, scale = 0.0;
          if (ss != 0.0) {
            const double nrm = sqrt(alpha * alpha + ss);
            beta = (alpha >= 0.0) ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            scale = 1.0 / (alpha - beta);
          }
          par[0] = tau; par[1] = beta; par[2] = scale;
        }
      }
      __syncthreads();
      const double tau = par[0], beta = par[1], scale = par[2];
      if (tid < BM) v[tid] = (tid == 0) ? 1.0 : (tid < m ? Ls[tid * LD] * scale : 0.0);
      __syncthreads();
      if (a.U) {
        const int64_t idx = uoff + k;
        if (tid < b) a.U[idx * b + tid] = v[tid];
        if (tid == 0) a.Utau[idx] = tau;
      }
      if (tid < m) Ls[tid * LD] = (tid == 0) ? beta : 0.0;
      if (tau != 0.0) {
        // TPR threads per row / column, each over every TPR-th index with two
        // accumulators, combined with lane shuffles (the TPR lanes sit in one warp)
        constexpr int TPR = BC_NT / BM;
        const int grp = tid / TPR, sub = tid % TPR;
        // left application to the rest of the bulge: columns 1 .. ncol-1
        {
          const int cc = 1 + grp;
          double d0 = 0.0, d1 = 0.0;
          if (cc < ncol) {
            int t = sub;
            for (; t + TPR < m; t += 2 * TPR) { d0 += v[t] * Ls[t * LD + cc]; d1 += v[t + TPR] * Ls[(t + TPR) * LD + cc]; }
            if (t < m) d0 += v[t] * Ls[t * LD + cc];
          }
          double dot = d0 + d1;
#pragma unroll
          for (int o = TPR / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
          if (cc < ncol) {
            dot *= tau;
            for (int t = sub; t < m; t += TPR) Ls[t * LD + cc] -= dot * v[t];
          }
        }
        // two-sided on the diagonal block: w = tau D v
        {
          const int p = grp;
          double d0 = 0.0, d1 = 0.0;
          if (p < m) {
            int q = sub;
            for (; q + TPR < m; q += 2 * TPR) { d0 += Ds[q * LD + p] * v[q]; d1 += Ds[(q + TPR) * LD + p] * v[q + TPR]; }
            if (q < m) d0 += Ds[q * LD + p] * v[q];
          }
          double dot = d0 + d1;
#pragma unroll
          for (int o = TPR / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
          if (p < m && sub == 0) wv[p] = tau * dot;
        }
        // right application to the block below
        {
          const int rr = grp;
          double d0 = 0.0, d1 = 0.0;
          if (rr < mb) {
            int t = sub;
            for (; t + TPR < m; t += 2 * TPR) { d0 += Bs[t * LD + rr] * v[t]; d1 += Bs[(t + TPR) * LD + rr] * v[t + TPR]; }
            if (t < m) d0 += Bs[t * LD + rr] * v[t];
          }
          double dot = d0 + d1;
#pragma unroll
          for (int o = TPR / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
          if (rr < mb) {
            dot *= tau;
            for (int t = sub; t < m; t += TPR) Bs[t * LD + rr] -= dot * v[t];
          }
        }
        __syncthreads();
        if (warp == 0) {
          double pv = 0.0;
          for (int t = lane; t < m; t += 32) pv += wv[t] * v[t];
          pv = warp_sum(pv);
          if (lane == 0) par[2] = 0.5 * tau * pv;
        }
        __syncthreads();
        const double alpha = par[2];
        if (tid < m) wv[tid] -= alpha * v[tid];
        __syncthreads();
        // rank-2 update of the lower triangle
        if (tr < m)
          for (int q = tc; q <= tr; q += CS) Ds[q * LD + tr] -= v[tr] * wv[q] + wv[tr] * v[q];
      }
      __syncthreads();
      // ---- write back
      if (tr < m) {
        for (int cc = tc; cc < ncol; cc += CS) bput(a.band, ldb, r0 + tr, c + cc, Ls[tr * LD + cc]);
        for (int q = tc; q <= tr; q += CS) bput(a.band, ldb, r0 + tr, r0 + q, Ds[q * LD + tr]);
      }
      if (tr < mb)
        for (int t = tc; t < m; t += CS) bput(a.band, ldb, r1 + 1 + tr, r0 + t, Bs[t * LD + tr]);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(a.prog + j, (int)(k + 1));
      }
    }
    if (K == 0 && tid == 0) st_release(a.prog + j, 0);
  }
}

// Carried, look-ahead form (b <= BM, NT = 4 BM threads).
//  * The block below written by step k, A(R_{k+1}, R_k), is exactly the left block
//    A(R_{k+1}, c' : r0'-1) of step k+1 (c' = r0 = r0' - b), and no other sweep
//    touches it in between, so it stays in shared memory: the two buffers swap
//    roles and the block is written back once, as step k+1's left block (or at the
//    sweep's end).
//  * Its first column is final once step k has applied its reflector from the
//    right, so warp 0 forms step k+1's reflector then, while the other warps finish
//    step k (the FP64 square root and divisions leave the critical path), and
//    stores step k+1's beta -- A(r0', c') -- to the band at once.
//  * Lag 2.  Sweep j step k touches the entries of sweep j-1 step k+2 only at that
//    step's beta entry (sweep j's block below reaches row r1 + b = r0' of sweep
//    j-1, column r1 = c').  Since beta is published within sweep j-1's step k+1,
//    sweep j step k may start as soon as sweep j-1 has completed step k+1; the
//    later write-back of the left block of step k+2 skips that entry, which sweep
//    j may already have updated.
//  * The symmetric mat-vec reads the lower triangle only; alpha = tau w^T v / 2
//    is formed by every warp, and w - alpha v once per entry.
// Same reflectors, same arithmetic per entry as the other forms up to the order
// of the dot-product partial sums.
template <int BM>
__global__ void __launch_bounds__(4 * BM, (BM <= 32) ? 4 : 2) k_bulge_chase_carry(const BcArgs a) {
  constexpr int NT = 4 * BM, TPR = 4, LD = BM + 1;
  extern __shared__ double smb[];
  double* Ds = smb;                 // Ds[q * LD + p] = A(r0 + p, r0 + q), p >= q
  double* buf0 = Ds + BM * LD;      // left block  L[cc * LD + t] = A(r0 + t, c + cc)
  double* buf1 = buf0 + BM * LD;    // block below B[t * LD + rr] = A(r1 + 1 + rr, r0 + t)
  __shared__ double vb0[BM], vb1[BM], wv[BM];
  __shared__ double par[4];         // [0] tau of this step, [1] tau of the next, [3] abort
  const int b = a.b, ldb = 2 * b + 1;
  const int64_t n = a.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid / TPR, sub = tid % TPR;
  for (int64_t j = blockIdx.x; j + 3 <= n; j += gridDim.x) {
    const int64_t K = sweep_steps(n, b, j);
    const int64_t Kprev = (j > 0) ? sweep_steps(n, b, j - 1) : 0;
    const int64_t uoff = sweep_offset(n, b, j);
    double* Ls = buf0;
    double* Bs = buf1;
    double* v = vb0;
    double* vn = vb1;
    for (int64_t k = 0; k < K; ++k) {
      if (j > 0) {
        int64_t need = k + BC_LAG_CARRY;
        if (need > Kprev) need = Kprev;
        if (tid == 0) par[3] = wait_geq(a.prog + (j - 1), (int)need, a.st, (int)(j + 1)) ? 0.0 : 1.0;
        __syncthreads();
        if (par[3] != 0.0) return;
      }
      const int64_t r0 = j + 1 + k * b;
      const int64_t r1 = (r0 + b - 1 < n - 1) ? r0 + b - 1 : n - 1;
      const int m = (int)(r1 - r0 + 1);
      const int64_t c = (k == 0) ? j : r0 - b;
      const int ncol = (int)(r0 - c);                                   // 1 for k = 0, b otherwise
      const int mb = (int)(((r1 + b < n - 1) ? r1 + b : n - 1) - r1);   // rows of the block below
      // ---- loads: diagonal block (lower), block below, and the left column at k = 0
#pragma unroll
      for (int it = 0; it < BM * BM / NT; ++it) {
        const int idx = tid + it * NT;
        const int p = idx % BM, q = idx / BM;
        if (p < m && q <= p) Ds[q * LD + p] = bget(a.band, ldb, r0 + p, r0 + q);
        if (p < mb && q < m) Bs[q * LD + p] = bget(a.band, ldb, r1 + 1 + p, r0 + q);
      }
      if (k == 0 && tid < m) Ls[tid] = bget(a.band, ldb, r0 + tid, c);
      __syncthreads();
      if (k == 0) {
        // ---- the first reflector of the sweep, from x = L(:, 0), by warp 0
        if (warp == 0) {
          double ss = 0.0;
          for (int t = 1 + lane; t < m; t += 32) { const double x = Ls[t]; ss += x * x; }
          ss = warp_sum(ss);
          const double alpha = Ls[0];
          double tau = 0.0, beta = alpha, scale = 0.0;
          if (ss != 0.0) {
            const double nrm = sqrt(alpha * alpha + ss);
            beta = (alpha >= 0.0) ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            scale = 1.0 / (alpha - beta);
          }
          for (int t = lane; t < BM; t += 32) {
            v[t] = (t == 0) ? 1.0 : (t < m ? Ls[t] * scale : 0.0);
            if (t < m) Ls[t] = (t == 0) ? beta : 0.0;
          }
          if (lane == 0) par[0] = tau;
          if (a.U) {
            for (int t = lane; t < b; t += 32) a.U[uoff * b + t] = v[t];
            if (lane == 0) a.Utau[uoff] = tau;
          }
        }
        __syncthreads();
      }
      const double tau = par[0];
      if (tau != 0.0) {
        // left application to the rest of the bulge: column cc = 1 + grp of L
        {
          const int cc = 1 + grp;
          double d0 = 0.0, d1 = 0.0;
          if (cc < ncol) {
            int t = sub;
            for (; t + TPR < m; t += 2 * TPR) { d0 += v[t] * Ls[cc * LD + t]; d1 += v[t + TPR] * Ls[cc * LD + t + TPR]; }
            if (t < m) d0 += v[t] * Ls[cc * LD + t];
          }
          double dot = d0 + d1;  // the shuffles run on every lane (converged warp)
          dot += __shfl_xor_sync(0xffffffffu, dot, 1);
          dot += __shfl_xor_sync(0xffffffffu, dot, 2);
          if (cc < ncol) {
            dot *= tau;
            for (int t2 = sub; t2 < m; t2 += TPR) Ls[cc * LD + t2] -= dot * v[t2];
          }
        }
        // w = tau D v from the lower triangle: row p = grp
        {
          const int p = grp;
          double d0 = 0.0;
          if (p < m) {
            for (int q = sub; q < m; q += TPR) d0 += ((q <= p) ? Ds[q * LD + p] : Ds[p * LD + q]) * v[q];
          }
          d0 += __shfl_xor_sync(0xffffffffu, d0, 1);
          d0 += __shfl_xor_sync(0xffffffffu, d0, 2);
          if (p < m && sub == 0) wv[p] = tau * d0;
        }
        // right application to the block below: row rr = grp
        {
          const int rr = grp;
          double d0 = 0.0, d1 = 0.0;
          if (rr < mb) {
            int t = sub;
            for (; t + TPR < m; t += 2 * TPR) { d0 += Bs[t * LD + rr] * v[t]; d1 += Bs[(t + TPR) * LD + rr] * v[t + TPR]; }
            if (t < m) d0 += Bs[t * LD + rr] * v[t];
          }
          double dot = d0 + d1;
          dot += __shfl_xor_sync(0xffffffffu, dot, 1);
          dot += __shfl_xor_sync(0xffffffffu, dot, 2);
          if (rr < mb) {
            dot *= tau;
            for (int t = sub; t < m; t += TPR) Bs[t * LD + rr] -= dot * v[t];
          }
        }
      }
      __syncthreads();
      const bool next = (k + 1 < K);
      if (tau != 0.0) {
        // w <- w - alpha v (alpha = tau w^T v / 2, formed by every warp)
        double pv = 0.0;
        for (int t = lane; t < m; t += 32) pv += wv[t] * v[t];
        pv = warp_sum(pv);
        const double alpha = 0.5 * tau * pv;
        __syncthreads();  // (every warp has read wv)
        if (tid < m) wv[tid] -= alpha * v[tid];
        __syncthreads();
      }
      if (warp == 0 && next) {
        // ---- look-ahead, while the other warps update the diagonal block: step
        // k+1's reflector from the final first column of the block below (the
        // rank-2 update does not touch that block); publish its beta entry now
        const int m1 = mb;
        double ss = 0.0;
        for (int t = 1 + lane; t < m1; t += 32) { const double x = Bs[t]; ss += x * x; }
        ss = warp_sum(ss);
        const double alpha = Bs[0];
        double tau1 = 0.0, beta = alpha, scale = 0.0;
        if (ss != 0.0) {
          const double nrm = sqrt(alpha * alpha + ss);
          beta = (alpha >= 0.0) ? -nrm : nrm;
          tau1 = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        for (int t = lane; t < BM; t += 32) {
          vn[t] = (t == 0) ? 1.0 : (t < m1 ? Bs[t] * scale : 0.0);
          if (t < m1) Bs[t] = (t == 0) ? beta : 0.0;
        }
        if (lane == 0) {
          par[1] = tau1;
          bput(a.band, ldb, r1 + 1, r0, beta);
        }
        if (a.U) {
          for (int t = lane; t < b; t += 32) a.U[(uoff + k + 1) * b + t] = vn[t];
          if (lane == 0) a.Utau[uoff + k + 1] = tau1;
        }
      } else if (tau != 0.0) {
        // the rank-2 update of the lower triangle, by every warp but the one forming
        // the next reflector
        const int t0 = next ? tid - 32 : tid, nt = next ? NT - 32 : NT;
        for (int idx = t0; idx < BM * BM; idx += nt) {
          const int p = idx % BM, q = idx / BM;
          if (p < m && q <= p) Ds[q * LD + p] -= v[p] * wv[q] + wv[p] * v[q];
        }
      }
      __syncthreads();
      // ---- write back the diagonal block and the left block (its beta entry was
      // published one step earlier, for k >= 1); the block below becomes the next
      // step's left block, or is written back at the sweep's end
#pragma unroll
      for (int it = 0; it < BM * BM / NT; ++it) {
        const int idx = tid + it * NT;
        const int p = idx % BM, q = idx / BM;
        if (p < m && q <= p) bput(a.band, ldb, r0 + p, r0 + q, Ds[q * LD + p]);
        if (p < m && q < ncol && (k == 0 || p != 0 || q != 0)) bput(a.band, ldb, r0 + p, c + q, Ls[q * LD + p]);
      }
      if (!next) {
#pragma unroll
        for (int it = 0; it < BM * BM / NT; ++it) {
          const int idx = tid + it * NT;
          const int p = idx % BM, q = idx / BM;
          if (p < mb && q < m) bput(a.band, ldb, r1 + 1 + p, r0 + q, Bs[q * LD + p]);
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(a.prog + j, (int)(k + 1));
        par[0] = par[1];
      }
      double* tmp = Ls; Ls = Bs; Bs = tmp;
      tmp = v; v = vn; vn = tmp;
    }
    if (K == 0 && tid == 0) st_release(a.prog + j, 0);
  }
}

__global__ void k_extract_tridiag(const double* band, int b, int64_t n, double* d, double* e) {
  const int ldb = 2 * b + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    d[i] = band[i * ldb];
    if (i + 1 < n) e[i] = (b >= 1) ? band[1 + i * ldb] : 0.0;
  }
}

}  // namespace

int64_t bc_num_reflectors(int64_t n, int b) {
  if (n < 3) return 0;
  return sweep_offset(n, b, n - 2);
}

evd_status_t bc_run(const PlanCore& pc, const BcWork& w, double* d, double* e, bool vectors) {
  const int64_t n = pc.n;
  cudaStream_t s = pc.stream;
  if (n >= 3 && pc.b >= 2) {
    EVD_CUDA_TRY(cudaMemsetAsync(w.prog, 0, sizeof(int) * n, s));
    BcArgs a;
    a.band = w.band; a.n = n; a.b = pc.b;
    a.U = vectors ? w.U : nullptr;
    a.Utau = w.Utau;
    a.prog = w.prog; a.st = pc.status;
    const void* kern = (const void*)k_bulge_chase;
    size_t smem = 0;
    int nt = BC_NT;
    const int variant = pc.bc_kernel;  // 0: global, 1: staged, 2: carried (default)
    if (variant >= 1 && pc.b <= 32) {
      kern = (variant == 2) ? (const void*)k_bulge_chase_carry<32> : (const void*)k_bulge_chase_smem<32>;
      smem = 3 * 32 * 33 * sizeof(double);
      nt = (variant == 2) ? 128 : BC_NT;
    } else if (variant >= 1 && pc.b <= 64) {
      kern = (variant == 2) ? (const void*)k_bulge_chase_carry<64> : (const void*)k_bulge_chase_smem<64>;
      smem = 3 * 64 * 65 * sizeof(double);
      nt = (variant == 2) ? 256 : BC_NT;
    }
    if (smem > 48 * 1024) {
      const evd_status_t st = ensure_dynamic_smem(kern, smem);
      if (st != EVD_OK) return st;
    }
    // Sweeps that can be in flight at once: a sweep of K steps starts about lag
    // steps after its predecessor, so about K / lag run together.  Two sweeps share
    // an SM only when there are more of those than SMs (sharing slows each sweep,
    // and below that the chain of sweeps sets the time).
    int maxG = max_coresident_blocks(kern, nt, smem);
    const int64_t inflight = (sweep_steps(n, pc.b, 0) + BC_LAG_CARRY - 1) / BC_LAG_CARRY;
    int per_sm = pc.bc_ctas_per_sm;
    if (per_sm <= 0) per_sm = (variant == 2 && inflight > (int64_t)pc.sms * 5 / 2) ? 2 : 1;
    if (pc.sms > 0 && maxG > pc.sms * per_sm) maxG = pc.sms * per_sm;
    // a CTA takes sweeps j = g, g + G, ...: sweep j + G may start once sweep j is
    // done, about K steps after its start, while the chain lets it start 2 G steps
    // after sweep j, so G a little above K / lag keeps every CTA busy; more CTAs
    // only take SMs that concurrent solves could use
    int64_t G = std::min<int64_t>(n - 2, inflight + inflight / 4 + 2);
    if (G > maxG) G = maxG;
    void* args[] = {&a};
    // model bytes (each step reads and writes its 2b x b window; U written once)
    const double nn = (double)n * (double)n;
    // FP64 flops: about 12 b^2 per step (left and right applications 4 b^2 each,
    // symmetric mat-vec 2 b^2, rank-2 update 2 b^2) over n^2 / (2b) steps
    StatScope sc("bc_chase", s, 6.0 * pc.b * nn, 16.0 * pc.b * nn + (vectors ? 4.0 * nn : 0.0));
    EVD_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(nt), args, smem, s)); count_launch();
  }
  if (n > 0) {
    k_extract_tridiag<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(w.band, pc.b, n, d, e); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
  }
  return EVD_OK;
}

}  // namespace evd
