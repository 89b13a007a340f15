// Batched Rayleigh-Ritz step of LOBPCG (Section 5.1): for every k-point the pencil (H, G) = (S^H Op S, S^H S) of
// its search space S = [X | W | P] (n <= 64 columns) is reduced to its m lowest Ritz pairs, one thread block per
// k-point, everything in shared memory, FP64.
//
//   1. unit-diagonal scaling D of G (a zero column gets D = 0 and is dropped below);
//   2. Cholesky of D G D with diagonal pivoting, stopped when the largest remaining pivot is below `drop`: the
//      retained pivot columns span the numerically independent part of span(S); rank r;
//   3. H3 = L^{-1} (D H D)_r L^{-H} by two forward substitutions (the second on Y^H = (L^{-1} H_r)^H);
//   4. Householder reduction of H3 to a real symmetric tridiagonal T (complex reflectors, then a diagonal phase
//      scaling makes the off-diagonal real and non-negative);
//   5. bisection on Sturm counts for the m lowest eigenvalues of T;
//   6. inverse iteration on T (partially pivoted tridiagonal LU, 3 steps), with modified Gram-Schmidt against
//      earlier members of the same cluster (eigenvalues closer than 1e-7 |T|), processed cluster position by
//      position so that members are orthogonal;
//   7. back-transformation y = Q Phi z, then coef = D P L^{-H} y.
//
// A GB300 SM retires about 2 FP64 FMA per clock, so one warp-wide FP64 instruction holds the FP64 unit of its SM
// sub-partition for tens of cycles and the kernel is bound by its count of FP64 warp instructions on the longest
// chain. Every phase is therefore spread over the block and over the four sub-partitions: substitutions
// column-oriented (one rank-1 row update per step for all threads), matrix-vector products split by rows and column
// quarters, the back-transformation for all wanted vectors at once (short shuffle trees per vector), shared
// matrices with an odd leading dimension (row-wise access by consecutive threads hits distinct banks), reciprocals
// and square roots of pivots taken once. Bisection (step 5) runs a group of 8 lanes per eigenvalue (multisection:
// each lane counts at one of 8 interior points), first in FP32 down to ~30 eps32 |T| (backward-stable Sturm counts
// make the FP32 bracket exact for a matrix within a few eps32 |T|; the bracket is widened by 16 eps32 |T| and
// verified by two FP64 counts, with the Gershgorin interval as fallback), then in FP64 to the absolute width
// eps64 |T| (LAPACK's default for bisection, below which the FP64 Sturm count itself is not accurate).
#include <cfloat>
#include <climits>
#include <cmath>

#include "pc_internal.cuh"

namespace pc {

namespace {

constexpr double RR_CLUSTER_REL = 1e-7;
constexpr int RR_MAXN = 64;
constexpr int RR_THREADS = 256;  // 8 warps: the Householder step splits its products over warp % 4 and warp / 4
constexpr double RR_EPS = 2.220446049250313e-16;

__device__ __forceinline__ double2 shfl_xor_d2(double2 v, int mask) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask));
}
__device__ __forceinline__ double2 warp_sum_d2(double2 v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = cadd(v, shfl_xor_d2(v, o));
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Partially pivoted LU of the tridiagonal (T - lam I), T = (d, e): factors in f[0..4r): 1/u0, u1, u2, l; pivots as
// 0/1 in f[4r..5r).
__device__ void tri_factor(const double *d, const double *e, int r, double lam, double tiny, double *f) {
  double *u0i = f, *u1 = f + r, *u2 = f + 2 * r, *l = f + 3 * r, *piv = f + 4 * r;
  double ca = d[0] - lam, cb = r > 1 ? e[0] : 0.0;
  for (int i = 0; i < r - 1; ++i) {
    const double sub = e[i];
    const double ai1 = d[i + 1] - lam, bi1 = (i + 1 < r - 1) ? e[i + 1] : 0.0;
    if (fabs(ca) >= fabs(sub)) {
      if (ca == 0.0) ca = tiny;
      const double ic = 1.0 / ca;
      l[i] = sub * ic;
      piv[i] = 0.0;
      u0i[i] = ic;
      u1[i] = cb;
      u2[i] = 0.0;
      ca = ai1 - l[i] * cb;
      cb = bi1;
    } else {
      const double is = 1.0 / sub;
      l[i] = ca * is;
      piv[i] = 1.0;
      u0i[i] = is;
      u1[i] = ai1;
      u2[i] = bi1;
      ca = cb - l[i] * ai1;
      cb = -l[i] * bi1;
    }
  }
  if (ca == 0.0) ca = tiny;
  u0i[r - 1] = 1.0 / ca;
}

__device__ void tri_solve(const double *f, int r, double *y) {
  const double *u0i = f, *u1 = f + r, *u2 = f + 2 * r, *l = f + 3 * r, *piv = f + 4 * r;
  for (int i = 0; i < r - 1; ++i) {
    if (piv[i] != 0.0) {
      const double yi = y[i];
      y[i] = y[i + 1];
      y[i + 1] = yi - l[i] * y[i + 1];
    } else {
      y[i + 1] -= l[i] * y[i];
    }
  }
  for (int i = r - 1; i >= 0; --i) {
    double s = y[i];
    if (i + 1 < r) s -= u1[i] * y[i + 1];
    if (i + 2 < r) s -= u2[i] * y[i + 2];
    y[i] = s * u0i[i];
  }
}

// number of eigenvalues of T = (d, e) below x (e2 = e^2), in the precision T of the arguments
template <typename R>
__device__ __forceinline__ int sturm_count(const R *d, const R *e2, int r, R x, R pivmin) {
  R q = d[0] - x;
  int c = q < R(0);
  for (int i = 1; i < r; ++i) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = d[i] - x - e2[i - 1] / q;
    c += q < R(0);
  }
  return c;
}

// FP64 version: the division by q is a multiplication by its correctly rounded reciprocal folded into one FMA, and
// the tests on q (sign, |q| < pivmin) read its bit pattern with integer instructions: 7 FP64 instructions a step
// instead of about 11. Each step still rounds with a relative error of a few ulp, which keeps the count backward
// stable (it is the exact count of a matrix whose d and e^2 differ from T's by a few ulp).
template <>
__device__ __forceinline__ int sturm_count<double>(const double *d, const double *e2, int r, double x, double pivmin) {
  const long long pm = __double_as_longlong(pivmin);
  double q = d[0] - x;
  long long qb = __double_as_longlong(q);
  int c = (qb < 0) & ((qb & LLONG_MAX) != 0);  // q < 0, -0.0 excluded
  for (int i = 1; i < r; ++i) {
    if ((qb & LLONG_MAX) < pm) q = -pivmin;
    q = fma(-e2[i - 1], __drcp_rn(q), d[i] - x);
    qb = __double_as_longlong(q);
    c += (qb < 0) & ((qb & LLONG_MAX) != 0);
  }
  return c;
}

// Multisection on a group of G lanes (G a power of two <= 32) per eigenvalue j: lane s of the group counts at the
// interior point lo + (s + 1) (hi - lo) / (G + 1); the leading run of lanes whose count is <= j gives the new bracket
// (the invariant count(lo) <= j < count(hi) holds whether or not the computed counts are monotone). All lanes of a
// group apply the same update. Runs while any group of the warp is still wider than its tolerance.
template <typename R>
__device__ void multisect(const R *d, const R *e2, int r, R pivmin, int j, int s, int G, bool active, R &lo, R &hi,
                          R atol, R rtol, int maxit) {
  const int lane = threadIdx.x & 31, base = lane & ~(G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  for (int it = 0; it < maxit; ++it) {
    const bool open = active && !(hi - lo <= fmax(atol, rtol * fmax(fabs(lo), fabs(hi))) + pivmin);
    if (!__any_sync(0xffffffffu, open)) break;
    const R step = (hi - lo) / R(G + 1);
    const R x = lo + R(s + 1) * step;
    const int c = open ? sturm_count<R>(d, e2, r, x, pivmin) : 0;
    const unsigned bits = (__ballot_sync(0xffffffffu, c <= j) >> base) & gmask;
    const int q = __ffs(~bits) - 1;  // leading lanes with count <= j (G when all)
    if (open) {
      const R nlo = q > 0 ? lo + R(q) * step : lo;
      const R nhi = q < G ? lo + R(q + 1) * step : hi;
      lo = nlo;
      hi = nhi;
    }
  }
}

__host__ __device__ inline int rr_ld(int n) { return (n & 1) ? n : n + 1; }

size_t rr_smem(int n, int m) {
  const int ld = rr_ld(n);
  return sizeof(double2) * (3 * (size_t)n * ld + 4 * (size_t)n + 4 * RR_MAXN) +
         sizeof(double) * (8 * (size_t)n + m) +
         sizeof(float) * 2 * (size_t)n + sizeof(int) * (2 * (size_t)n + m) + 64;
}

__global__ void __launch_bounds__(RR_THREADS) rr_kernel(const double2 *__restrict__ Gg, const double2 *__restrict__ Hg,
                                                        int n, int m, double drop, double *__restrict__ thetag,
                                                        double2 *__restrict__ coefg, int *__restrict__ rankg,
                                                        const int *__restrict__ act, long sg, long sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LD = rr_ld(n);
  double2 *A = reinterpret_cast<double2 *>(smem_raw);  // scaled G -> pivoted Cholesky factor (lower)
  double2 *B = A + n * LD;                              // scaled H -> H3 -> tridiagonal; then Z (real r x m)
  double2 *Vh = B + n * LD;                             // Householder vectors, row k = v_k
  double2 *phi = Vh + n * LD;                           // phases of the tridiagonal scaling
  double2 *pv = phi + n;                                // p / q vectors of the Householder step
  double2 *vv = pv + n;                                 // Householder vectors: two buffers (look-ahead)
  double2 *vv2 = vv + n;
  double2 *hpart = vv2 + n;                             // partial products of a Householder step [4][RR_MAXN]
  double *dsc = reinterpret_cast<double *>(hpart + 4 * RR_MAXN);
  double *dd = dsc + n, *ee = dd + n, *e2 = ee + n, *tau = e2 + n, *dinv = tau + n, *w = dinv + n;  // w: m
  double *spare = w + m;                                                                              // 2n
  float *d32 = reinterpret_cast<float *>(spare + 2 * n);
  float *e232 = d32 + n;
  int *perm = reinterpret_cast<int *>(e232 + n);
  int *pos = perm + n;  // m
  __shared__ int s_p, s_r, s_stop, s_maxpos;
  __shared__ double s_il, s_lkk, s_tau2[2], s_gl, s_gu, s_tn, s_pivmin;
  __shared__ double2 s_alpha2[2], s_Kp[2];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int b = act ? act[blockIdx.x] : (int)blockIdx.x;
  const double2 *G = Gg + (long)b * sg;
  const double2 *H = Hg + (long)b * sg;
  double *Z = reinterpret_cast<double *>(B);

  // 1. scaling
  for (int i = tid; i < n; i += nt) {
    const double gii = G[i * n + i].x;
    dsc[i] = gii > 0.0 ? 1.0 / sqrt(gii) : 0.0;
    perm[i] = i;
  }
  __syncthreads();
  for (int i = tid; i < n * n; i += nt) {
    const int r = i / n, c = i - r * n;
    const double f = dsc[r] * dsc[c];
    const double2 x = G[r * n + c], y = G[c * n + r];
    A[r * LD + c] = cmake<double2>(0.5 * (x.x + y.x) * f, 0.5 * (x.y - y.y) * f);
    const double2 u = H[r * n + c], v = H[c * n + r];
    B[r * LD + c] = cmake<double2>(0.5 * (u.x + v.x) * f, 0.5 * (u.y - v.y) * f);
  }
  if (tid == 0) s_r = n;
  __syncthreads();

  // 2. pivoted Cholesky
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      // pivot: the largest remaining diagonal entry. Non-negative doubles order like their bit patterns read as
      // signed 64-bit integers (negative ones fall below all of them), so the search costs no FP64 instructions;
      // the pivot's square root and its reciprocal are formed once, by lane 0
      long long best = LLONG_MIN;
      int bi = n;
      for (int i = k + lane; i < n; i += 32) {
        const long long v = __double_as_longlong(A[i * LD + i].x);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        const double piv = bi < n ? __longlong_as_double(best) : -1.0;
        s_p = bi < n ? bi : k;
        s_stop = !(piv > drop);
        if (s_stop) {
          s_r = k;
        } else {
          const double il = rsqrt(piv);
          s_il = il;
          s_lkk = piv * il;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != k) {
      for (int c = tid; c < n; c += nt) {
        double2 t = A[k * LD + c];
        A[k * LD + c] = A[p * LD + c];
        A[p * LD + c] = t;
        t = B[k * LD + c];
        B[k * LD + c] = B[p * LD + c];
        B[p * LD + c] = t;
      }
      __syncthreads();
      for (int r = tid; r < n; r += nt) {
        double2 t = A[r * LD + k];
        A[r * LD + k] = A[r * LD + p];
        A[r * LD + p] = t;
        t = B[r * LD + k];
        B[r * LD + k] = B[r * LD + p];
        B[r * LD + p] = t;
      }
      if (tid == 0) {
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
      }
      __syncthreads();
    }
    const double il = s_il;
    for (int i = k + 1 + tid; i < n; i += nt) A[i * LD + k] = cscale(A[i * LD + k], il);
    __syncthreads();
    if (tid == 0) A[k * LD + k] = cmake<double2>(s_lkk, 0.0);
    const int t = n - k - 1;
    for (int e = tid; e < t * t; e += nt) {
      const int q = e / t, i = k + 1 + q, j = k + 1 + e - q * t;
      const double2 a = A[i * LD + k], c = A[j * LD + k];
      double2 v = A[i * LD + j];  // v -= a conj(c): four FP64 FMA
      v.x = fma(-a.x, c.x, fma(-a.y, c.y, v.x));
      v.y = fma(-a.y, c.x, fma(a.x, c.y, v.y));
      A[i * LD + j] = v;
    }
    __syncthreads();
  }
  const int r = s_r;
  for (int i = tid; i < r; i += nt) dinv[i] = 1.0 / A[i * LD + i].x;
  __syncthreads();
  // unit lower factor U = L diag(1/L_ii) (column i scaled by 1/L_ii) into Vh, free until step 4
  for (int e = tid; e < r * r; e += nt) {
    const int kk = e / r, i = e - kk * r;
    if (i < kk) Vh[kk * LD + i] = cscale(A[kk * LD + i], dinv[i]);
  }
  __syncthreads();

  // 3. H3 = L^{-1} H_r L^{-H}: two column-oriented forward substitutions with U (row i, once final, updates all rows
  // below it: four FP64 FMA per entry; the rows are scaled by 1/L_ii at the end), a conjugate transpose in between
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i + 1 < r; ++i) {
      const int below = r - i - 1;
      for (int e = tid; e < below * r; e += nt) {
        const int q = e / r, kk = i + 1 + q, j = e - q * r;
        const double2 c = Vh[kk * LD + i], y = B[i * LD + j];
        double2 v = B[kk * LD + j];
        v.x = fma(-c.x, y.x, fma(c.y, y.y, v.x));
        v.y = fma(-c.x, y.y, fma(-c.y, y.x, v.y));
        B[kk * LD + j] = v;
      }
      __syncthreads();
    }
    for (int e = tid; e < r * r; e += nt) {
      const int i = e / r, j = e % r;
      B[i * LD + j] = cscale(B[i * LD + j], dinv[i]);
    }
    __syncthreads();
    if (pass == 0) {
      for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e % r;
        if (i < j) {
          const double2 x = B[i * LD + j], y = B[j * LD + i];
          B[i * LD + j] = cmake<double2>(y.x, -y.y);
          B[j * LD + i] = cmake<double2>(x.x, -x.y);
        } else if (i == j) {
          B[i * LD + i].y = -B[i * LD + i].y;
        }
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e % r;
    if (i < j) {
      const double2 x = B[i * LD + j], y = B[j * LD + i];
      const double2 h = cmake<double2>(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
      B[i * LD + j] = h;
      B[j * LD + i] = cmake<double2>(h.x, -h.y);
    } else if (i == j) {
      B[i * LD + i].y = 0.0;
    }
  }
  __syncthreads();

  // 4. Householder tridiagonalisation of H3 (r x r), on its lower triangle. A GB300 SM retires about 2 FP64 FMA
  // per clock, so one warp-wide FP64 instruction holds an SM sub-partition's FP64 unit for tens of cycles: every
  // step below keeps its chains of FP64 instructions short and spreads its products over all four sub-partitions.
  // Look-ahead: in the rank-2 update of step k, warp 0 updates the trailing block's first column first and forms
  // the reflector of step k+1 from it while the other warps update the rest, so the reflector's serial chain of
  // scalar FP64 work overlaps the update (two reflector buffers alternate).
  //
  // reflector of column kk (warp 0): x = B[kk+1:, kk], sigma = |x|^2; v = x - alpha e1, alpha = -phase(x0) |x|,
  // tau = 2 / |v|^2 with |v|^2 = 2 (sigma + |x0| |x|) (no cancellation)
  auto make_reflector = [&](int kk, double2 *vb, int slot) {
    const int tt = r - kk - 1;
    double sig = 0.0;
    for (int i = lane; i < tt; i += 32) {
      const double2 x = B[(kk + 1 + i) * LD + kk];
      vb[i] = x;
      sig = fma(x.x, x.x, fma(x.y, x.y, sig));
    }
    sig = warp_sum_d(sig);
    if (lane == 0) {
      const double2 x0 = vb[0];
      if (sig == 0.0) {
        s_tau2[slot] = 0.0;
      } else {
        const double a0 = fma(x0.x, x0.x, x0.y * x0.y);
        const double nrm = sig * rsqrt(sig);
        double2 ph = cmake<double2>(1.0, 0.0);
        double ax0 = 0.0;
        if (a0 > 0.0) {
          const double ra = rsqrt(a0);
          ax0 = a0 * ra;
          ph = cmake<double2>(x0.x * ra, x0.y * ra);
        }
        s_alpha2[slot] = cmake<double2>(-ph.x * nrm, -ph.y * nrm);
        vb[0] = cmake<double2>(fma(ph.x, nrm, x0.x), fma(ph.y, nrm, x0.y));
        s_tau2[slot] = 1.0 / fma(nrm, ax0, sig);
      }
    }
  };
  // B_sub -= v q^H + q v^H at entry (i, j) of the trailing block of step k: eight FP64 FMA
  auto rank2_entry = [&](int k, int i, int j, const double2 *vc) {
    const double2 vi = vc[i], qi = pv[i], vj = vc[j], qj = pv[j];
    double2 *bp = B + (k + 1 + i) * LD + k + 1 + j;
    double2 bv = *bp;
    bv.x = fma(-vi.x, qj.x, fma(-vi.y, qj.y, fma(-qi.x, vj.x, fma(-qi.y, vj.y, bv.x))));
    bv.y = fma(-vi.y, qj.x, fma(vi.x, qj.y, fma(-qi.y, vj.x, fma(qi.x, vj.y, bv.y))));
    *bp = bv;
  };
  int cur = 0;        // reflector buffer of the current step
  bool have = false;  // its reflector was formed by the previous step's look-ahead
  for (int k = 0; k + 2 < r; ++k) {
    const int t = r - k - 1;
    double2 *vc = cur ? vv2 : vv;
    if (!have) {
      if (warp == 0) make_reflector(k, vc, cur);
      __syncthreads();
    }
    const double tk = s_tau2[cur];
    if (tid == 0) tau[k] = tk;
    if (tk == 0.0) {
      for (int i = tid; i < t; i += nt) Vh[k * LD + i] = cmake<double2>(0.0, 0.0);
      __syncthreads();
      have = false;
      continue;
    }
    // partial products of B_sub v from the lower triangle of B_sub (the only part kept up to date): warp w takes
    // rows 32 (w / 4) + lane and the quarter w % 4 of the columns; entry j <= i from row i, j > i as the conjugate of
    // column i (the conjugation flips a sign bit, no FP64 work). Consecutive rows hit distinct banks (LD odd),
    // column reads are contiguous.
    {
      const int c = warp & 3, i = (warp >> 2) * 32 + lane;
      const int cl = (t + 3) >> 2, j0 = c * cl, j1 = min(t, j0 + cl);
      if (i < t) {
        const double2 *row = B + (k + 1 + i) * LD + k + 1;
        const double2 *col = B + (k + 1) * LD + k + 1 + i;
        double2 s = cmake<double2>(0.0, 0.0);
        for (int j = j0; j < j1; ++j) {
          double2 a = j <= i ? row[j] : col[j * LD];
          a.y = __longlong_as_double(__double_as_longlong(a.y) ^ ((long long)(j > i) << 63));
          const double2 x = vc[j];
          s.x = fma(a.x, x.x, fma(-a.y, x.y, s.x));
          s.y = fma(a.x, x.y, fma(a.y, x.x, s.y));
        }
        hpart[c * RR_MAXN + i] = s;
      }
    }
    __syncthreads();
    // p = tau B_sub v, K = tau/2 v^H p, q = p - K v on the row warps (two when t > 32, joined by a named barrier)
    if (warp == 0 || (warp == 1 && t > 32)) {
      const int i = tid;
      double2 p = cmake<double2>(0.0, 0.0), w = p;
      if (i < t) {
        p = cscale(cadd(cadd(hpart[i], hpart[RR_MAXN + i]), cadd(hpart[2 * RR_MAXN + i], hpart[3 * RR_MAXN + i])),
                   tk);
        Vh[k * LD + i] = vc[i];
        w = cmulc(vc[i], p);
      }
      w = warp_sum_d2(w);
      if (lane == 0) s_Kp[warp] = w;
      if (t > 32)
        asm volatile("bar.sync 1, 64;" ::: "memory");
      else
        __syncwarp();
      double2 K = s_Kp[0];
      if (t > 32) K = cadd(K, s_Kp[1]);
      K = cscale(K, 0.5 * tk);
      if (i < t) pv[i] = csub(p, cmul(K, vc[i]));
    }
    __syncthreads();
    // the rank-2 update on the lower triangle, entries packed row by row (e -> (i, j), j <= i) so that every warp
    // is full; with a next step, warp 0 takes the first column and the next reflector, warps 1.. the entries j >= 1
    const bool ahead = k + 3 < r;
    if (ahead && warp == 0) {
      for (int i = lane; i < t; i += 32) rank2_entry(k, i, 0, vc);
      __syncwarp();
      make_reflector(k + 1, cur ? vv : vv2, 1 - cur);
    }
    {
      const int off = ahead ? 1 : 0, first = ahead ? 32 : 0, nthr = nt - first, tt = t - off;
      if (tid >= first)
        for (int e = tid - first; e < tt * (tt + 1) / 2; e += nthr) {
          int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
          if (i * (i + 1) / 2 > e) --i;
          if ((i + 1) * (i + 2) / 2 <= e) ++i;
          const int j = e - i * (i + 1) / 2;
          rank2_entry(k, i + off, j + off, vc);
        }
      for (int i = tid; i < t; i += nt) B[(k + 1 + i) * LD + k] = i == 0 ? s_alpha2[cur] : cmake<double2>(0.0, 0.0);
    }
    __syncthreads();
    have = ahead;
    if (ahead) cur = 1 - cur;
  }

  // real tridiagonal T = Phi^H T_c Phi: moduli and unit phases in parallel, the phase product on one thread
  for (int i = tid; i < r; i += nt) {
    dd[i] = B[i * LD + i].x;
    d32[i] = (float)dd[i];
    if (i + 1 < r) {
      const double2 c = B[(i + 1) * LD + i];
      const double ac = hypot(c.x, c.y);
      ee[i] = ac;
      e2[i] = ac * ac;
      e232[i] = (float)(ac * ac);
      pv[i] = ac > 0.0 ? cmake<double2>(c.x / ac, c.y / ac) : cmake<double2>(1.0, 0.0);
    }
  }
  __syncthreads();
  if (warp == 0) {
    double gl = HUGE_VAL, gu = -HUGE_VAL, tn = 0.0, emax2 = 0.0;
    for (int i = lane; i < r; i += 32) {
      const double off = (i > 0 ? ee[i - 1] : 0.0) + (i + 1 < r ? ee[i] : 0.0);
      gl = fmin(gl, dd[i] - off);
      gu = fmax(gu, dd[i] + off);
      tn = fmax(tn, fabs(dd[i]) + off);
      if (i + 1 < r) emax2 = fmax(emax2, e2[i]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
      gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
      tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
      emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
    }
    if (lane == 0) {
      const double pm = 1e-300 * fmax(1.0, emax2);
      s_pivmin = pm;
      s_tn = tn;
      s_gl = gl - RR_EPS * 2.0 * tn - pm;
      s_gu = gu + RR_EPS * 2.0 * tn + pm;
    }
  } else if (tid == 32) {
    phi[0] = cmake<double2>(1.0, 0.0);
    for (int i = 0; i + 1 < r; ++i) phi[i + 1] = cmul(phi[i], pv[i]);
  }
  __syncthreads();

  // 5. bisection: eigenvalue j (ascending) of T on a group of G lanes (G = 8 up to 32 wanted eigenvalues)
  const int mm = m < r ? m : r;
  {
    const int G = mm <= nt / 8 ? 8 : (mm <= nt / 4 ? 4 : (mm <= nt / 2 ? 2 : 1));
    if (tid < ((mm * G + 31) & ~31)) {
      const int j = tid / G, s = tid % G, base = (tid & 31) & ~(G - 1);
      const bool active = j < mm;
      const int jj = active ? j : 0;
      const double tn = s_tn, pivmin = s_pivmin;
      // FP32 bracket
      const float tn32 = (float)tn;
      const float pivmin32 = 1e-30f * fmaxf(1.0f, tn32 * tn32);
      float lo32 = (float)s_gl, hi32 = (float)s_gu;
      lo32 -= fabsf(lo32) * 1e-6f + FLT_MIN;
      hi32 += fabsf(hi32) * 1e-6f + FLT_MIN;
      multisect<float>(d32, e232, r, pivmin32, jj, s, G, active, lo32, hi32, 32.0f * FLT_EPSILON * tn32, 0.0f, 60);
      // widen, verify in FP64 (lanes 0 and 1 of the group count at the ends), fall back to the Gershgorin interval
      const double margin = 16.0 * FLT_EPSILON * tn + pivmin;
      double lo = (double)lo32 - margin, hi = (double)hi32 + margin;
      const int cnt = (active && s < 2) ? sturm_count<double>(dd, e2, r, s == 0 ? lo : hi, pivmin) : 0;
      const int clo = __shfl_sync(0xffffffffu, cnt, base), chi = __shfl_sync(0xffffffffu, cnt, base + (G > 1 ? 1 : 0));
      const int chi1 = G > 1 ? chi : (active ? sturm_count<double>(dd, e2, r, hi, pivmin) : 0);
      if (!(clo <= jj && chi1 > jj)) {
        lo = s_gl;
        hi = s_gu;
      }
      multisect<double>(dd, e2, r, pivmin, jj, s, G, active, lo, hi, RR_EPS * tn, 2.0 * RR_EPS, 200);
      if (active && s == 0) w[j] = 0.5 * (lo + hi);
    }
  }
  __syncthreads();
  if (tid == 0) {
    int mp = 0;
    for (int j = 0; j < mm; ++j) {
      pos[j] = (j > 0 && w[j] - w[j - 1] <= RR_CLUSTER_REL * s_tn) ? pos[j - 1] + 1 : 0;
      mp = pos[j] > mp ? pos[j] : mp;
    }
    s_maxpos = mp;
  }
  __syncthreads();

  // 6. inverse iteration, cluster position by cluster position; Z (r x mm, column-major by j) lives in B
  const int maxpos = s_maxpos;
  // eigenvector j on warp j % 4, lane j / 4: the sequential solves run on all four SM sub-partitions
  for (int round = 0; round <= maxpos; ++round) {
    for (int j = warp + 4 * lane; warp < 4 && j < mm; j += 128) {
      if (pos[j] != round) continue;
      double work[5 * RR_MAXN];
      double *z = Z + (long)j * r;
      tri_factor(dd, ee, r, w[j], RR_EPS * s_tn + 1e-300, work);
      for (int i = 0; i < r; ++i) {  // a fixed start vector with no special structure
        const unsigned hsh = (unsigned)i * 2654435761u + (unsigned)j * 40503u + 12345u;
        z[i] = 1.0 + 0.37 * ((double)((hsh >> 12) & 1023u) / 512.0 - 1.0);
      }
      for (int step = 0; step < 3; ++step) {
        tri_solve(work, r, z);
        for (int q = j - pos[j]; q < j; ++q) {  // earlier members of the cluster
          const double *zq = Z + (long)q * r;
          double dot = 0.0;
          for (int i = 0; i < r; ++i) dot += zq[i] * z[i];
          for (int i = 0; i < r; ++i) z[i] -= dot * zq[i];
        }
        double nrm = 0.0;
        for (int i = 0; i < r; ++i) nrm += z[i] * z[i];
        nrm = 1.0 / sqrt(nrm);
        for (int i = 0; i < r; ++i) z[i] *= nrm;
      }
    }
    __syncthreads();
  }

  // 7. back-transformation y = Q Phi z (reflectors applied last to first), then L^H x = y, coef = D P x.
  double2 *out = coefg + (long)b * sc;
  // Block-parallel form for all wanted vectors at once when the work space fits behind Z in B: Y (r x mm, row
  // stride YLD odd, so that a column read by consecutive rows hits distinct banks) and the reflector coefficients s
  // (mm). The coefficient s_j of a reflector is summed by a group of C consecutive lanes (rows c, c + C, ...) and a
  // shuffle tree: one barrier per reflector step instead of two, a reduction depth of log2 C instead of C.
  const long zsz = ((long)r * mm + 1) / 2;
  const int YLD = mm | 1;
  int C = 1;
  while (2 * C <= 32 && 2 * C * mm <= nt) C *= 2;
  if (mm > 0 && zsz + (long)r * YLD + mm <= (long)n * LD) {
    double2 *Y = B + zsz, *sj = Y + (long)r * YLD;
    for (int e = tid; e < r * mm; e += nt) {
      const int i = e / mm, j = e - i * mm;
      Y[(long)i * YLD + j] = cscale(phi[i], Z[(long)j * r + i]);
    }
    __syncthreads();
    for (int k = r - 3; k >= 0; --k) {
      const double tk = tau[k];
      if (tk == 0.0) continue;  // uniform over the block
      const int t = r - k - 1;
      // s_j = tau v_k^H Y[k+1:, j]
      if (tid < ((C * mm + 31) & ~31)) {  // whole warps (the shuffles)
        const int j = tid / C, c = tid - j * C;
        double2 acc = cmake<double2>(0.0, 0.0);
        if (j < mm)
          for (int i = c; i < t; i += C) {
            const double2 v = Vh[k * LD + i], y = Y[(long)(k + 1 + i) * YLD + j];  // acc += conj(v) y
            acc.x = fma(v.x, y.x, fma(v.y, y.y, acc.x));
            acc.y = fma(v.x, y.y, fma(-v.y, y.x, acc.y));
          }
        for (int o = C >> 1; o; o >>= 1) acc = cadd(acc, shfl_xor_d2(acc, o));
        if (j < mm && c == 0) sj[j] = cscale(acc, tk);
      }
      __syncthreads();
      for (int e = tid; e < t * mm; e += nt) {
        const int i = e / mm, j = e - i * mm;
        const double2 v = Vh[k * LD + i], sv = sj[j];  // Y -= v s
        double2 y = Y[(long)(k + 1 + i) * YLD + j];
        y.x = fma(-v.x, sv.x, fma(v.y, sv.y, y.x));
        y.y = fma(-v.x, sv.y, fma(-v.y, sv.x, y.y));
        Y[(long)(k + 1 + i) * YLD + j] = y;
      }
      __syncthreads();
    }
    // L^H x = y, column-oriented from the last row: row i, final once all rows below have been applied, updates the
    // rows above it (the scaling by 1/L_ii is applied to row i at the end). The coefficients L_il / L_ii go to Vh
    // (free now) first, so that the update is four FP64 FMA per entry.
    for (int e = tid; e < r * r; e += nt) {
      const int i = e / r, l = e - i * r;
      if (l < i) Vh[i * LD + l] = cscale(A[i * LD + l], dinv[i]);
    }
    __syncthreads();
    for (int i = r - 1; i > 0; --i) {
      for (int e = tid; e < i * mm; e += nt) {
        const int l = e / mm, j = e - l * mm;
        const double2 c = Vh[i * LD + l], y = Y[(long)i * YLD + j];  // Y[l] -= conj(c) Y[i]
        double2 v = Y[(long)l * YLD + j];
        v.x = fma(-c.x, y.x, fma(-c.y, y.y, v.x));
        v.y = fma(-c.x, y.y, fma(c.y, y.x, v.y));
        Y[(long)l * YLD + j] = v;
      }
      __syncthreads();
    }
    for (int e = tid; e < n * m; e += nt) out[e] = cmake<double2>(0.0, 0.0);
    __syncthreads();
    for (int e = tid; e < r * mm; e += nt) {
      const int i = e / mm, j = e - i * mm;
      out[perm[i] * m + j] = cscale(Y[(long)i * YLD + j], dinv[i] * dsc[perm[i]]);
    }
    for (int j = tid; j < m; j += nt) thetag[(long)b * m + j] = j < mm ? w[j] : 0.0;
    if (rankg && tid == 0) rankg[b] = r;
    return;
  }
  // Otherwise one warp per Ritz vector held in registers (lane l owns rows l and l + 32).
  for (int j = warp; j < m; j += nwarp) {
    double2 y0 = cmake<double2>(0.0, 0.0), y1 = y0;
    const int i0 = lane, i1 = lane + 32;
    if (j < mm) {
      const double *z = Z + (long)j * r;
      if (i0 < r) y0 = cscale(phi[i0], z[i0]);
      if (i1 < r) y1 = cscale(phi[i1], z[i1]);
      for (int k = r - 3; k >= 0; --k) {
        const double tk = tau[k];
        if (tk == 0.0) continue;
        // rows k+1 .. r-1 hold v_k[row - k - 1]
        double2 s = cmake<double2>(0.0, 0.0);
        if (i0 > k && i0 < r) s = cadd(s, cmulc(Vh[k * LD + i0 - k - 1], y0));
        if (i1 > k && i1 < r) s = cadd(s, cmulc(Vh[k * LD + i1 - k - 1], y1));
        s = cscale(warp_sum_d2(s), tk);
        if (i0 > k && i0 < r) y0 = csub(y0, cmul(Vh[k * LD + i0 - k - 1], s));
        if (i1 > k && i1 < r) y1 = csub(y1, cmul(Vh[k * LD + i1 - k - 1], s));
      }
      // L^H x = y (upper triangular), rows from the last
      for (int i = r - 1; i >= 0; --i) {
        double2 s = cmake<double2>(0.0, 0.0);
        if (i0 > i && i0 < r) s = cadd(s, cmulc(A[i0 * LD + i], y0));
        if (i1 > i && i1 < r) s = cadd(s, cmulc(A[i1 * LD + i], y1));
        s = warp_sum_d2(s);
        if (i0 == i) y0 = cscale(csub(y0, s), dinv[i]);
        if (i1 == i) y1 = cscale(csub(y1, s), dinv[i]);
      }
    }
    for (int i = lane; i < n; i += 32) out[i * m + j] = cmake<double2>(0.0, 0.0);
    __syncwarp();
    if (j < mm) {
      if (i0 < r) out[perm[i0] * m + j] = cscale(y0, dsc[perm[i0]]);
      if (i1 < r) out[perm[i1] * m + j] = cscale(y1, dsc[perm[i1]]);
    }
    if (lane == 0) thetag[(long)b * m + j] = j < mm ? w[j] : 0.0;
  }
  if (rankg && tid == 0) rankg[b] = r;
}

}  // namespace

double rr_flops(int n, int m) {
  const double c = (double)n * n * n;
  // complex multiply-adds: Cholesky n^3/6, the two substitutions 2 x n^3/2, tridiagonalisation 2n^3/3 (matrix-vector
  // product and rank-2 update per step), back-transformation 3 n^2 m / 2; 8 real flops each
  return 8.0 * (c / 6.0 + c + 2.0 * c / 3.0 + 1.5 * (double)n * n * m);
}

int launch_rr(int nb, int n, int m, const void *G, const void *H, double drop, double *theta, void *coef, int *rank,
              cudaStream_t st, const int *act, long sg, long sc) {
  if (nb == 0) return PC_OK;
  if (n > RR_MAXN || m > n) {
    set_error("rayleigh_ritz: need m <= n <= %d", RR_MAXN);
    return PC_EINVAL;
  }
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(rr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rr_smem(RR_MAXN, RR_MAXN)));
    configured = true;
  }
  rr_kernel<<<nb, RR_THREADS, rr_smem(n, m), st>>>(static_cast<const double2 *>(G), static_cast<const double2 *>(H),
                                                    n, m, drop, theta, static_cast<double2 *>(coef), rank, act,
                                                    sg > 0 ? sg : (long)n * n, sc > 0 ? sc : (long)n * m);
  PC_CK_LAUNCH();
  return PC_OK;
}

}  // namespace pc
