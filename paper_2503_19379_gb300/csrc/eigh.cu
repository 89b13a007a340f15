// Small dense FP64 Hermitian eigensolver (two-sided cyclic Jacobi) and the Rayleigh-Ritz step of LOBPCG
// (Section 5.1), one thread block per k-point, everything in shared memory.
//
// Jacobi: the n(n-1)/2 index pairs are visited in round-robin order, n/2 disjoint pairs at a time. For a pair (p,q)
// with a_pq = |a_pq| e^{i phi}, the unitary U = diag(1, e^{-i phi}) [[c, s], [-s, c]] makes the 2x2 block diagonal,
// with tau = (a_qq - a_pp) / (2 |a_pq|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c
// (the symmetric 2x2 Schur rotation, applied after removing the phase). All pairs of one step are applied at once
// as A <- U^H (A U). A pair is skipped when |a_pq| <= 1e-15 sqrt(|a_pp a_qq|) (relative to the pair's diagonal, which
// keeps the small eigenvalues of positive definite matrices accurate) or |a_pq| <= 1e-14 |a_qq - a_pp| (rotation
// angle below 1e-14); sweeps stop when a sweep skips every pair (at most 40).
#include <cmath>

#include "pc_internal.cuh"

namespace pc {

constexpr int JAC_MAX_SWEEPS = 40;
constexpr double JAC_REL_TOL = 1e-15;
constexpr double JAC_ANGLE_TOL = 1e-14;

struct JacScratch {
  double c[32], s[32];
  double2 e[32];
  int p[32], q[32];
  int any;
};

// Eigen-decomposition of the Hermitian n x n matrix in A (leading dimension ld, row-major); on return the
// eigenvalues (ascending) are in w[0..n) and V (leading dimension ld) holds the eigenvectors in columns, in the
// same order. A is destroyed. Uses `tmp` (n doubles + n ints worth of shared space) for sorting.
__device__ void jacobi_eigh(double2 *A, double2 *V, int n, int ld, double *w, int *rankbuf, double2 *colbuf,
                            JacScratch *js) {
  const int P = n + (n & 1);
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int r = i / n, c = i - r * n;
    V[r * ld + c] = cmake<double2>(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  if (n == 1) {
    if (threadIdx.x == 0) w[0] = A[0].x;
    __syncthreads();
    return;
  }
  for (int sweep = 0; sweep < JAC_MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) js->any = 0;
    __syncthreads();
    for (int rnd = 0; rnd < P - 1; ++rnd) {
      // 1. rotation parameters of the P/2 disjoint pairs of this round (circle method, player P-1 fixed)
      for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
        int p, q;
        if (t == 0) {
          p = rnd;
          q = P - 1;
        } else {
          p = (rnd + t) % (P - 1);
          q = (rnd - t + P - 1) % (P - 1);
        }
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        double c = 1.0, s = 0.0;
        double2 e = cmake<double2>(1.0, 0.0);
        if (q < n) {
          const double app = A[p * ld + p].x, aqq = A[q * ld + q].x;
          const double2 apq = A[p * ld + q];
          const double mag = hypot(apq.x, apq.y);
          // negligible when small relative to the geometric mean of the diagonal (near-degenerate pairs) or when
          // the rotation angle |a_pq| / |a_qq - a_pp| is below 1e-14 (well-separated pairs: the eigenvalue moves by
          // |a_pq|^2 / |a_qq - a_pp|)
          if (mag > JAC_REL_TOL * sqrt(fabs(app * aqq)) && mag > JAC_ANGLE_TOL * fabs(aqq - app) && mag > 1e-300) {
            const double tau = (aqq - app) / (2.0 * mag);
            const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
            e = cmake<double2>(apq.x / mag, -apq.y / mag);  // e^{-i phi}
            js->any = 1;
          } else {
            q = n;  // mark as identity
          }
        }
        js->p[t] = p;
        js->q[t] = q;
        js->c[t] = c;
        js->s[t] = s;
        js->e[t] = e;
      }
      __syncthreads();
      // 2. columns: A <- A U, V <- V U
      for (int it = threadIdx.x; it < n * (P / 2); it += blockDim.x) {
        const int t = it / n, k = it - t * n;
        const int p = js->p[t], q = js->q[t];
        if (q >= n) continue;
        const double c = js->c[t], s = js->s[t];
        const double2 e = js->e[t];
        {
          const double2 akp = A[k * ld + p], akq = A[k * ld + q];
          const double2 eq = cmul(e, akq);
          A[k * ld + p] = cmake<double2>(c * akp.x - s * eq.x, c * akp.y - s * eq.y);
          A[k * ld + q] = cmake<double2>(s * akp.x + c * eq.x, s * akp.y + c * eq.y);
        }
        {
          const double2 vkp = V[k * ld + p], vkq = V[k * ld + q];
          const double2 eq = cmul(e, vkq);
          V[k * ld + p] = cmake<double2>(c * vkp.x - s * eq.x, c * vkp.y - s * eq.y);
          V[k * ld + q] = cmake<double2>(s * vkp.x + c * eq.x, s * vkp.y + c * eq.y);
        }
      }
      __syncthreads();
      // 3. rows: A <- U^H A
      for (int it = threadIdx.x; it < n * (P / 2); it += blockDim.x) {
        const int t = it / n, k = it - t * n;
        const int p = js->p[t], q = js->q[t];
        if (q >= n) continue;
        const double c = js->c[t], s = js->s[t];
        const double2 e = js->e[t];
        const double2 apk = A[p * ld + k], aqk = A[q * ld + k];
        const double2 eq = cmulc(e, aqk);  // conj(e) * a_qk
        A[p * ld + k] = cmake<double2>(c * apk.x - s * eq.x, c * apk.y - s * eq.y);
        A[q * ld + k] = cmake<double2>(s * apk.x + c * eq.x, s * apk.y + c * eq.y);
      }
      __syncthreads();
    }
    const int any = js->any;
    __syncthreads();
    if (!any) break;
  }
  // sort ascending: rank by counting, then permute V's columns through colbuf
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double wi = A[i * ld + i].x;
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const double wj = A[j * ld + j].x;
      r += (wj < wi) || (wj == wi && j < i);
    }
    rankbuf[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[rankbuf[i]] = A[i * ld + i].x;
  for (int row = 0; row < n; ++row) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) colbuf[rankbuf[i]] = V[row * ld + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) V[row * ld + i] = colbuf[i];
    __syncthreads();
  }
}

constexpr int EIGH_MAXN = 64;

__global__ void __launch_bounds__(256) eigh_batched_kernel(const double2 *__restrict__ Ag, double *__restrict__ wg,
                                                          double2 *__restrict__ Vg, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *A = reinterpret_cast<double2 *>(smem_raw);
  double2 *V = A + n * n;
  double2 *colbuf = V + n * n;
  double *w = reinterpret_cast<double *>(colbuf + n);
  int *rankbuf = reinterpret_cast<int *>(w + n);
  __shared__ JacScratch js;
  const int b = blockIdx.x;
  const double2 *a = Ag + (long)b * n * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int r = i / n, c = i - r * n;
    const double2 x = a[r * n + c], y = a[c * n + r];
    A[i] = cmake<double2>(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
  }
  __syncthreads();
  jacobi_eigh(A, V, n, n, w, rankbuf, colbuf, &js);
  for (int i = threadIdx.x; i < n; i += blockDim.x) wg[(long)b * n + i] = w[i];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) Vg[(long)b * n * n + i] = V[i];
}

// Rayleigh-Ritz for one pencil (H, G), n x n, wanted m. grid = nb (active), 256 threads.
// Shared: A, V, C (n x n each), colbuf, w, d, rank.
__global__ void __launch_bounds__(256) rr_kernel(const double2 *__restrict__ Gg, const double2 *__restrict__ Hg, int n,
                                                int m, double drop, double *__restrict__ thetag,
                                                double2 *__restrict__ coefg, int *__restrict__ rankg,
                                                const int *__restrict__ act) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *A = reinterpret_cast<double2 *>(smem_raw);
  double2 *V = A + n * n;
  double2 *Cm = V + n * n;
  double2 *colbuf = Cm + n * n;
  double *w = reinterpret_cast<double *>(colbuf + n);
  double *dsc = w + n;
  int *rankbuf = reinterpret_cast<int *>(dsc + n);
  __shared__ JacScratch js;
  __shared__ int s_r;
  const int b = act ? act[blockIdx.x] : (int)blockIdx.x;
  const double2 *G = Gg + (long)b * n * n;
  const double2 *H = Hg + (long)b * n * n;

  // 1. unit-diagonal scaling of G
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double gii = G[i * n + i].x;
    dsc[i] = gii > 0.0 ? 1.0 / sqrt(gii) : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int r = i / n, c = i - r * n;
    const double2 x = G[r * n + c], y = G[c * n + r];
    const double f = dsc[r] * dsc[c];
    A[i] = cmake<double2>(0.5 * (x.x + y.x) * f, 0.5 * (x.y - y.y) * f);
  }
  __syncthreads();
  // 2. first orthonormalisation pass: C1 = D V_k w_k^{-1/2} over the retained (largest) eigenvalues
  jacobi_eigh(A, V, n, n, w, rankbuf, colbuf, &js);
  if (threadIdx.x == 0) {
    const double wmax = w[n - 1];
    int r = 0;
    for (int i = 0; i < n; ++i) r += (w[i] > drop * wmax);
    s_r = r;
  }
  __syncthreads();
  const int r = s_r;
  const int off = n - r;
  for (int i = threadIdx.x; i < n * r; i += blockDim.x) {
    const int row = i / r, col = i - row * r;
    const double f = dsc[row] / sqrt(w[off + col]);
    const double2 v = V[row * n + off + col];
    Cm[row * n + col] = cmake<double2>(v.x * f, v.y * f);
  }
  __syncthreads();
  // 3. second pass: G2 = C1^H G C1 (r x r); V <- G C1 first
  for (int i = threadIdx.x; i < n * r; i += blockDim.x) {
    const int row = i / r, col = i - row * r;
    double2 acc = cmake<double2>(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
      const double2 x = G[row * n + k], y = G[k * n + row];
      const double2 g = cmake<double2>(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
      acc = cadd(acc, cmul(g, Cm[k * n + col]));
    }
    V[row * n + col] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) {
    const int row = i / r, col = i - row * r;
    double2 acc = cmake<double2>(0.0, 0.0);
    for (int k = 0; k < n; ++k) acc = cadd(acc, cmulc(Cm[k * n + row], V[k * n + col]));
    A[row * r + col] = acc;
  }
  __syncthreads();
  jacobi_eigh(A, V, r, r, w, rankbuf, colbuf, &js);
  // C <- C1 V2 w2^{-1/2}, through A as temporary (n x r)
  for (int i = threadIdx.x; i < n * r; i += blockDim.x) {
    const int row = i / r, col = i - row * r;
    double2 acc = cmake<double2>(0.0, 0.0);
    for (int k = 0; k < r; ++k) acc = cadd(acc, cmul(Cm[row * n + k], V[k * r + col]));
    const double f = 1.0 / sqrt(w[col]);
    A[row * n + col] = cmake<double2>(acc.x * f, acc.y * f);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * r; i += blockDim.x) {
    const int row = i / r, col = i - row * r;
    Cm[row * n + col] = A[row * n + col];
  }
  __syncthreads();
  // 4. projected operator H2 = C^H H C; V <- H C first
  for (int i = threadIdx.x; i < n * r; i += blockDim.x) {
    const int row = i / r, col = i - row * r;
    double2 acc = cmake<double2>(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
      const double2 x = H[row * n + k], y = H[k * n + row];
      const double2 h = cmake<double2>(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
      acc = cadd(acc, cmul(h, Cm[k * n + col]));
    }
    V[row * n + col] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) {
    const int row = i / r, col = i - row * r;
    double2 acc = cmake<double2>(0.0, 0.0);
    for (int k = 0; k < n; ++k) acc = cadd(acc, cmulc(Cm[k * n + row], V[k * n + col]));
    A[row * r + col] = acc;
  }
  __syncthreads();
  jacobi_eigh(A, V, r, r, w, rankbuf, colbuf, &js);
  // 5. outputs: the lowest m Ritz values and coef = C U[:, :m] (zero columns if r < m)
  for (int i = threadIdx.x; i < m; i += blockDim.x) thetag[(long)b * m + i] = i < r ? w[i] : 0.0;
  for (int i = threadIdx.x; i < n * m; i += blockDim.x) {
    const int row = i / m, col = i - row * m;
    double2 acc = cmake<double2>(0.0, 0.0);
    if (col < r)
      for (int k = 0; k < r; ++k) acc = cadd(acc, cmul(Cm[row * n + k], V[k * r + col]));
    coefg[(long)b * n * m + i] = acc;
  }
  if (rankg && threadIdx.x == 0) rankg[b] = r;
}

// ------------------------------------------------------------------------------------------------ fast Rayleigh-Ritz
// The same Rayleigh-Ritz as rr_kernel with far fewer FP64 operations (a single SM runs FP64 at ~8 GFLOP/s):
//   1. unit-diagonal scaling D of G (a zero column gets D = 0 and is dropped below);
//   2. Cholesky of D G D with diagonal pivoting, stopped when the largest remaining pivot is below `drop`: the
//      retained pivot columns span the numerically independent part of span(S); rank r;
//   3. H3 = L^{-1} (D H D)_r L^{-H} by two forward substitutions (the second on Y^H = (L^{-1} H_r)^H);
//   4. Householder reduction of H3 to a real symmetric tridiagonal T (complex reflectors, then a diagonal phase
//      scaling makes the off-diagonal real and non-negative);
//   5. bisection on Sturm counts for the m lowest eigenvalues of T (one thread per eigenvalue);
//   6. inverse iteration on T (partially pivoted tridiagonal LU, 3 steps), with modified Gram-Schmidt against
//      earlier members of the same cluster (eigenvalues closer than 1e-7 |T|), processed cluster position by
//      position so that members are orthogonal;
//   7. back-transformation through the phases and the reflectors, and coef = D P L^{-H} y.
constexpr double RR_CLUSTER_REL = 1e-7;
constexpr int RR_MAXN = 64;

// partially pivoted LU of the tridiagonal (T - lam I), T = (d, e); factors in f[0..4r): u0, u1, u2, l; pivots as
// 0/1 in f[4r..5r)
__device__ void tri_factor(const double *d, const double *e, int r, double lam, double tiny, double *f) {
  double *u0 = f, *u1 = f + r, *u2 = f + 2 * r, *l = f + 3 * r, *piv = f + 4 * r;
  double ca = d[0] - lam, cb = r > 1 ? e[0] : 0.0;
  for (int i = 0; i < r - 1; ++i) {
    const double sub = e[i];
    const double ai1 = d[i + 1] - lam, bi1 = (i + 1 < r - 1) ? e[i + 1] : 0.0;
    if (fabs(ca) >= fabs(sub)) {
      if (ca == 0.0) ca = tiny;
      l[i] = sub / ca;
      piv[i] = 0.0;
      u0[i] = ca;
      u1[i] = cb;
      u2[i] = 0.0;
      ca = ai1 - l[i] * cb;
      cb = bi1;
    } else {
      l[i] = ca / sub;
      piv[i] = 1.0;
      u0[i] = sub;
      u1[i] = ai1;
      u2[i] = bi1;
      ca = cb - l[i] * ai1;
      cb = -l[i] * bi1;
    }
  }
  if (ca == 0.0) ca = tiny;
  u0[r - 1] = ca;
}

__device__ void tri_solve(const double *f, int r, double *y) {
  const double *u0 = f, *u1 = f + r, *u2 = f + 2 * r, *l = f + 3 * r, *piv = f + 4 * r;
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
    y[i] = s / u0[i];
  }
}

__device__ int sturm_count(const double *d, const double *e, int r, double x, double pivmin) {
  double q = d[0] - x;
  int c = q < 0.0;
  for (int i = 1; i < r; ++i) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    c += q < 0.0;
  }
  return c;
}

static size_t rr2_smem(int n, int m) {
  return sizeof(double2) * (3 * (size_t)n * n + 3 * (size_t)n) + sizeof(double) * (6 * (size_t)n + m) +
         sizeof(int) * (2 * (size_t)n + m);
}

__global__ void __launch_bounds__(256) rr2_kernel(const double2 *__restrict__ Gg, const double2 *__restrict__ Hg,
                                                 int n, int m, double drop, double *__restrict__ thetag,
                                                 double2 *__restrict__ coefg, int *__restrict__ rankg,
                                                 const int *__restrict__ act) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *A = reinterpret_cast<double2 *>(smem_raw);  // scaled G -> pivoted Cholesky factor (lower)
  double2 *B = A + n * n;                               // scaled H -> Y -> H3 -> tridiagonal; then Z (real r x m)
  double2 *Vh = B + n * n;                              // Householder vectors, row k = v_k
  double2 *phi = Vh + n * n;                            // phases of the tridiagonal scaling
  double2 *pv = phi + n;                                // p / q vectors of the Householder step
  double2 *vv = pv + n;                                 // current Householder vector
  double *dsc = reinterpret_cast<double *>(vv + n);
  double *dd = dsc + n, *ee = dd + n, *tau = ee + n, *w = tau + n, *misc = w + m;  // misc: n doubles
  int *perm = reinterpret_cast<int *>(misc + n);
  int *pos = perm + n;
  int *pcount = pos + m;  // n ints (unused padding for alignment safety)
  (void)pcount;
  __shared__ int s_p, s_r, s_stop;
  __shared__ double s_piv, s_tau, s_gl, s_gu, s_tn, s_pivmin;
  __shared__ double2 s_alpha, s_K;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int b = act ? act[blockIdx.x] : (int)blockIdx.x;
  const double2 *G = Gg + (long)b * n * n;
  const double2 *H = Hg + (long)b * n * n;
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
    A[i] = cmake<double2>(0.5 * (x.x + y.x) * f, 0.5 * (x.y - y.y) * f);
    const double2 u = H[r * n + c], v = H[c * n + r];
    B[i] = cmake<double2>(0.5 * (u.x + v.x) * f, 0.5 * (u.y - v.y) * f);
  }
  if (tid == 0) s_r = n;
  __syncthreads();
  // 2. pivoted Cholesky
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      int p = k;
      double best = A[k * n + k].x;
      for (int i = k + 1; i < n; ++i)
        if (A[i * n + i].x > best) {
          best = A[i * n + i].x;
          p = i;
        }
      s_p = p;
      s_piv = best;
      s_stop = !(best > drop);
      if (s_stop) s_r = k;
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != k) {
      for (int c = tid; c < n; c += nt) {
        double2 t = A[k * n + c];
        A[k * n + c] = A[p * n + c];
        A[p * n + c] = t;
        t = B[k * n + c];
        B[k * n + c] = B[p * n + c];
        B[p * n + c] = t;
      }
      __syncthreads();
      for (int r = tid; r < n; r += nt) {
        double2 t = A[r * n + k];
        A[r * n + k] = A[r * n + p];
        A[r * n + p] = t;
        t = B[r * n + k];
        B[r * n + k] = B[r * n + p];
        B[r * n + p] = t;
      }
      if (tid == 0) {
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
      }
      __syncthreads();
    }
    const double lkk = sqrt(s_piv);
    for (int i = k + 1 + tid; i < n; i += nt) A[i * n + k] = cscale(A[i * n + k], 1.0 / lkk);
    __syncthreads();
    if (tid == 0) A[k * n + k] = cmake<double2>(lkk, 0.0);
    const int t = n - k - 1;
    for (int e = tid; e < t * t; e += nt) {
      const int i = k + 1 + e / t, j = k + 1 + e % t;
      const double2 a = A[i * n + k], c = A[j * n + k];
      A[i * n + j] = csub(A[i * n + j], cmake<double2>(a.x * c.x + a.y * c.y, a.y * c.x - a.x * c.y));
    }
    __syncthreads();
  }
  const int r = s_r;
  // 3. H3 = L^{-1} H_r L^{-H}: forward substitution on H_r, conjugate transpose, forward substitution again
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < r; ++i) {
      for (int j = tid; j < r; j += nt) {
        double2 s = B[i * n + j];
        for (int k = 0; k < i; ++k) s = csub(s, cmul(A[i * n + k], B[k * n + j]));
        B[i * n + j] = cscale(s, 1.0 / A[i * n + i].x);
      }
      __syncthreads();
    }
    if (pass == 0) {
      for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e % r;
        if (i < j) {
          const double2 x = B[i * n + j], y = B[j * n + i];
          B[i * n + j] = cmake<double2>(y.x, -y.y);
          B[j * n + i] = cmake<double2>(x.x, -x.y);
        } else if (i == j) {
          B[i * n + i].y = -B[i * n + i].y;
        }
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e % r;
    if (i < j) {
      const double2 x = B[i * n + j], y = B[j * n + i];
      const double2 h = cmake<double2>(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
      B[i * n + j] = h;
      B[j * n + i] = cmake<double2>(h.x, -h.y);
    } else if (i == j) {
      B[i * n + i].y = 0.0;
    }
  }
  __syncthreads();
  // 4. Householder tridiagonalisation of H3 (r x r, leading dimension n)
  for (int k = 0; k + 2 < r; ++k) {
    const int t = r - k - 1;
    if (tid == 0) {
      double sig = 0.0;
      for (int i = 0; i < t; ++i) {
        const double2 x = B[(k + 1 + i) * n + k];
        sig += x.x * x.x + x.y * x.y;
      }
      const double2 x0 = B[(k + 1) * n + k];
      const double ax0 = hypot(x0.x, x0.y);
      if (sig == 0.0) {
        s_tau = 0.0;
      } else {
        const double2 ph = ax0 > 0.0 ? cmake<double2>(x0.x / ax0, x0.y / ax0) : cmake<double2>(1.0, 0.0);
        const double nrm = sqrt(sig);
        s_alpha = cmake<double2>(-ph.x * nrm, -ph.y * nrm);
        const double2 v0 = csub(x0, s_alpha);
        const double vn2 = sig - ax0 * ax0 + v0.x * v0.x + v0.y * v0.y;
        s_tau = 2.0 / vn2;
        vv[0] = v0;
      }
    }
    __syncthreads();
    const double tk = s_tau;
    if (tid == 0) tau[k] = tk;
    if (tk == 0.0) {
      for (int i = tid; i < t; i += nt) Vh[k * n + i] = cmake<double2>(0.0, 0.0);
      __syncthreads();
      continue;
    }
    for (int i = 1 + tid; i < t; i += nt) vv[i] = B[(k + 1 + i) * n + k];
    __syncthreads();
    for (int i = tid; i < t; i += nt) {
      Vh[k * n + i] = vv[i];
      double2 s = cmake<double2>(0.0, 0.0);
      for (int j = 0; j < t; ++j) s = cadd(s, cmul(B[(k + 1 + i) * n + k + 1 + j], vv[j]));
      pv[i] = cscale(s, tk);
    }
    __syncthreads();
    if (tid == 0) {
      double2 s = cmake<double2>(0.0, 0.0);
      for (int i = 0; i < t; ++i) s = cadd(s, cmulc(vv[i], pv[i]));
      s_K = cscale(s, 0.5 * tk);
    }
    __syncthreads();
    const double2 K = s_K;
    for (int i = tid; i < t; i += nt) pv[i] = csub(pv[i], cmul(K, vv[i]));
    __syncthreads();
    for (int e = tid; e < t * t; e += nt) {
      const int i = e / t, j = e % t;
      const double2 vi = vv[i], qi = pv[i], vj = vv[j], qj = pv[j];
      // v_i conj(q_j) + q_i conj(v_j)
      const double2 upd = cadd(cmake<double2>(vi.x * qj.x + vi.y * qj.y, vi.y * qj.x - vi.x * qj.y),
                               cmake<double2>(qi.x * vj.x + qi.y * vj.y, qi.y * vj.x - qi.x * vj.y));
      B[(k + 1 + i) * n + k + 1 + j] = csub(B[(k + 1 + i) * n + k + 1 + j], upd);
    }
    for (int i = tid; i < t; i += nt) {
      const double2 val = i == 0 ? s_alpha : cmake<double2>(0.0, 0.0);
      B[(k + 1 + i) * n + k] = val;
      B[k * n + k + 1 + i] = cmake<double2>(val.x, -val.y);
    }
    __syncthreads();
  }
  // real tridiagonal T = Phi^H T_c Phi and its Gershgorin interval
  if (tid == 0) {
    phi[0] = cmake<double2>(1.0, 0.0);
    double gl = 1e300, gu = -1e300, tn = 0.0, emax2 = 0.0;
    for (int i = 0; i < r; ++i) dd[i] = B[i * n + i].x;
    for (int i = 0; i + 1 < r; ++i) {
      const double2 c = B[(i + 1) * n + i];
      const double ac = hypot(c.x, c.y);
      ee[i] = ac;
      phi[i + 1] = ac > 0.0 ? cmul(phi[i], cmake<double2>(c.x / ac, c.y / ac)) : phi[i];
      emax2 = fmax(emax2, ac * ac);
    }
    for (int i = 0; i < r; ++i) {
      const double off = (i > 0 ? ee[i - 1] : 0.0) + (i + 1 < r ? ee[i] : 0.0);
      gl = fmin(gl, dd[i] - off);
      gu = fmax(gu, dd[i] + off);
      tn = fmax(tn, fabs(dd[i]) + off);
    }
    const double pm = 1e-300 * fmax(1.0, emax2);
    s_pivmin = pm;
    s_tn = tn;
    s_gl = gl - 2.2e-16 * 2.0 * tn - pm;
    s_gu = gu + 2.2e-16 * 2.0 * tn + pm;
  }
  __syncthreads();
  // 5. bisection: eigenvalue j (ascending) of T
  const int mm = m < r ? m : r;
  for (int j = tid; j < mm; j += nt) {
    double lo = s_gl, hi = s_gu;
    for (int it = 0; it < 200; ++it) {
      if (hi - lo <= 2.2e-16 * 2.0 * fmax(fabs(lo), fabs(hi)) + s_pivmin) break;
      const double mid = 0.5 * (lo + hi);
      if (sturm_count(dd, ee, r, mid, s_pivmin) > j) hi = mid;
      else lo = mid;
    }
    w[j] = 0.5 * (lo + hi);
  }
  __syncthreads();
  if (tid == 0) {
    int mp = 0;
    for (int j = 0; j < mm; ++j) {
      pos[j] = (j > 0 && w[j] - w[j - 1] <= RR_CLUSTER_REL * s_tn) ? pos[j - 1] + 1 : 0;
      mp = pos[j] > mp ? pos[j] : mp;
    }
    s_p = mp;
  }
  __syncthreads();
  // 6. inverse iteration, cluster position by cluster position; Z (r x mm, column-major by j) lives in B
  const int maxpos = s_p;
  double2 work2[3 * RR_MAXN];  // per-thread: tridiagonal LU factors (5 r doubles), later y (r complex)
  double *work = reinterpret_cast<double *>(work2);
  for (int round = 0; round <= maxpos; ++round) {
    for (int j = tid; j < mm; j += nt) {
      if (pos[j] != round) continue;
      double *z = Z + (long)j * r;
      tri_factor(dd, ee, r, w[j], 2.2e-16 * s_tn + 1e-300, work);
      for (int i = 0; i < r; ++i) z[i] = 1.0 + 0.37 * sin(1.3 * i + 0.7 * j);
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
  // 7. back-transformation y = Q Phi z, then coef = D P L^{-H} y, one thread per wanted column
  for (int j = tid; j < m; j += nt) {
    double2 *y = work2;
    if (j < mm) {
      const double *z = Z + (long)j * r;
      for (int i = 0; i < r; ++i) y[i] = cscale(phi[i], z[i]);
      for (int k = r - 3; k >= 0; --k) {
        const double tk = tau[k];
        if (tk == 0.0) continue;
        const int t = r - k - 1;
        double2 s = cmake<double2>(0.0, 0.0);
        for (int i = 0; i < t; ++i) s = cadd(s, cmulc(Vh[k * n + i], y[k + 1 + i]));
        s = cscale(s, tk);
        for (int i = 0; i < t; ++i) y[k + 1 + i] = csub(y[k + 1 + i], cmul(Vh[k * n + i], s));
      }
      // L^H x = y (upper triangular, back substitution)
      for (int i = r - 1; i >= 0; --i) {
        double2 s = y[i];
        for (int k2 = i + 1; k2 < r; ++k2) s = csub(s, cmulc(A[k2 * n + i], y[k2]));
        y[i] = cscale(s, 1.0 / A[i * n + i].x);
      }
    }
    double2 *out = coefg + (long)b * n * m;
    for (int i = 0; i < n; ++i) out[i * m + j] = cmake<double2>(0.0, 0.0);
    if (j < mm)
      for (int i = 0; i < r; ++i) out[perm[i] * m + j] = cscale(y[i], dsc[perm[i]]);
    thetag[(long)b * m + j] = j < mm ? w[j] : 0.0;
  }
  if (rankg && tid == 0) rankg[b] = r;
}

static size_t rr_smem(int n) { return sizeof(double2) * (3 * (size_t)n * n + n) + sizeof(double) * 2 * n + sizeof(int) * n; }
static size_t eigh_smem(int n) { return sizeof(double2) * (2 * (size_t)n * n + n) + sizeof(double) * n + sizeof(int) * n; }

int launch_rr(int nb, int n, int m, const void *G, const void *H, double drop, double *theta, void *coef, int *rank,
              cudaStream_t st, const int *act) {
  if (nb == 0) return PC_OK;
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(rr2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rr2_smem(RR_MAXN, RR_MAXN)));
    configured = true;
  }
  rr2_kernel<<<nb, 256, rr2_smem(n, m), st>>>(static_cast<const double2 *>(G), static_cast<const double2 *>(H), n, m,
                                              drop, theta, static_cast<double2 *>(coef), rank, act);
  PC_CK_LAUNCH();
  return PC_OK;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_eigh_batched(int nb, int n, const void *A, double *w, void *V, void *stream) {
  PC_REQUIRE(A && w && V, "pc_eigh_batched: null argument");
  PC_REQUIRE(nb >= 0 && n >= 1 && n <= EIGH_MAXN, "pc_eigh_batched: need 1 <= n <= %d", EIGH_MAXN);
  if (nb == 0) return PC_OK;
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(eigh_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)eigh_smem(EIGH_MAXN)));
    configured = true;
  }
  eigh_batched_kernel<<<nb, 256, eigh_smem(n), (cudaStream_t)stream>>>(static_cast<const double2 *>(A), w,
                                                                         static_cast<double2 *>(V), n);
  PC_CK_LAUNCH();
  return PC_OK;
}

extern "C" int pc_rayleigh_ritz(int nb, int n, int m, const void *G, const void *H, double drop, double *theta,
                                void *coef, int *rank, void *stream) {
  PC_REQUIRE(G && H && theta && coef, "pc_rayleigh_ritz: null argument");
  PC_REQUIRE(nb >= 0 && n >= 1 && n <= EIGH_MAXN && m >= 1 && m <= n, "pc_rayleigh_ritz: bad sizes n=%d m=%d", n, m);
  PC_REQUIRE(drop >= 0.0 && drop < 1.0, "pc_rayleigh_ritz: drop must be in [0, 1)");
  return launch_rr(nb, n, m, G, H, drop, theta, coef, rank, (cudaStream_t)stream, nullptr);
}
