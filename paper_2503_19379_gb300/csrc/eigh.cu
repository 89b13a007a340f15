// Small dense FP64 Hermitian eigensolver (two-sided cyclic Jacobi), one thread block per matrix, everything in
// shared memory; and the C entry point of the Rayleigh-Ritz step (rr.cu).
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

static size_t eigh_smem(int n) { return sizeof(double2) * (2 * (size_t)n * n + n) + sizeof(double) * n + sizeof(int) * n; }

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
