// Learned warm start for the block eigensolver: forward, backward and Adam kernels of a small 3D convolutional
// network that predicts the initial block X0 (nb face fields) and guesses of log lambda from M0 = 1/eps and the
// Bloch vector k. The paper starts LOBPCG from a random block and has no network; the model is defined here:
//   conv1  3 -> C1 = 8 channels, 3x3x3, stride 2, circular padding, bias, ReLU           (N/2)^3
//   conv2  C1 -> C2 = 16, the same form                                                      (N/4)^3
//   FiLM   z = (1 + Fa phi + fa) relu(a2) + (Fc phi + fc), phi = (sin k, cos k)
//   head   1x1x1, C2 -> 6 nb channels (band, component, re/im): the coarse block
//   upsampling x4 per axis by periodic linear interpolation to the N^3 face grid: X0
//   value  y = Wv [mean z; phi] + bv
// Loss of one sample with converged eigenvectors V (orthonormal): nb - tr(G^{-1} B B^H), G = X^H X, B = X^H V (the
// principal-angle distance of span X to span V), plus w (y - log lambda)^2 per band. Its gradient in X is
// X C1 + V C2 with C1 = 2 G^{-1} B B^H G^{-1}, C2 = -2 B^H G^{-1}; the Grams and the two products run on this
// library's Gram and block-update kernels. Everything else is FP32 on the CUDA cores: the network is small (5352
// parameters at nb = 8) and its layers move a few MB per sample, so each kernel is bound by memory traffic or
// latency, not arithmetic. Weight gradients are sums over all samples and points, reduced inside one thread block
// per output entry group in a fixed order (deterministic, no atomics).
//
// Parameters: one flat float array in the order W1 (C1,3,3,3,3), b1, W2 (C2,C1,3,3,3), b2, Fa (C2,6), fa,
// Fc (C2,6), fc, Wh (6nb,C2), bh, Wv (nb,C2+6), bv, each row-major.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pc_internal.cuh"

namespace pc {
namespace ws {

constexpr int C1 = PC_WS_C1, C2 = PC_WS_C2, NBMAX = 16, TPB = 256;

struct Offs {
  long W1, b1, W2, b2, Fa, fa, Fc, fc, Wh, bh, Wv, bv, total;
};

Offs offsets(int nb) {
  Offs o;
  long p = 0;
  o.W1 = p, p += C1 * 3 * 27;
  o.b1 = p, p += C1;
  o.W2 = p, p += C2 * C1 * 27;
  o.b2 = p, p += C2;
  o.Fa = p, p += C2 * 6;
  o.fa = p, p += C2;
  o.Fc = p, p += C2 * 6;
  o.fc = p, p += C2;
  o.Wh = p, p += 6 * nb * C2;
  o.bh = p, p += 6 * nb;
  o.Wv = p, p += nb * (C2 + 6);
  o.bv = p, p += nb;
  o.total = p;
  return o;
}

// device workspace of one forward + backward pass over S samples (offsets in bytes, 256-aligned)
struct Work {
  size_t phi, a1, a2, z, pool, dy, coarse, G, B, Cx, Cv, dX, dcoarse, dz, da2, da1, dsa, dsc, loss, gram, total;
};

Work work_layout(int N, int nb, int S) {
  const long n1 = (long)(N / 2) * (N / 2) * (N / 2), m3 = (long)(N / 4) * (N / 4) * (N / 4);
  const long L = 3L * N * N * N;
  Work w;
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p += (bytes + 255) / 256 * 256;
    return at;
  };
  w.phi = take(sizeof(float) * 6 * S);
  w.a1 = take(sizeof(float) * (size_t)S * C1 * n1);
  w.a2 = take(sizeof(float) * (size_t)S * C2 * m3);
  w.z = take(sizeof(float) * (size_t)S * C2 * m3);
  w.pool = take(sizeof(float) * (size_t)S * C2);
  w.dy = take(sizeof(float) * (size_t)S * nb);
  w.coarse = take(sizeof(float2) * (size_t)S * nb * 3 * m3);
  w.G = take(sizeof(double2) * (size_t)S * nb * nb);
  w.B = take(sizeof(double2) * (size_t)S * nb * nb);
  w.Cx = take(sizeof(double2) * (size_t)S * nb * nb);
  w.Cv = take(sizeof(double2) * (size_t)S * nb * nb);
  w.dX = take(sizeof(float2) * (size_t)S * nb * L);
  w.dcoarse = take(sizeof(float2) * (size_t)S * nb * 3 * m3);
  w.dz = take(sizeof(float) * (size_t)S * C2 * m3);
  w.da2 = take(sizeof(float) * (size_t)S * C2 * m3);
  w.da1 = take(sizeof(float) * (size_t)S * C1 * n1);
  w.dsa = take(sizeof(float) * (size_t)S * C2);
  w.dsc = take(sizeof(float) * (size_t)S * C2);
  w.loss = take(sizeof(double) * (size_t)S);
  w.gram = take(std::max<size_t>(16, gram_scratch_bytes(S, L, nb, nb)));
  w.total = p;
  return w;
}

// ------------------------------------------------------------------------------------------------------- forward
// Stride-2 3x3x3 circular convolution: out[s][o][q] = b[o] + sum_{c,d} W[o][c][d] in[s][c][2q + d - 1 mod n].
// The input of conv1 is M0 of structure sidx[s] (3 channels); that of conv2 is relu(a1). grid (ceil(nout / 256), S)
template <int CIN, int COUT, bool RELU_IN>
__global__ void __launch_bounds__(TPB) conv_fwd_kernel(const float *__restrict__ in, long in_stride,
                                                       const int *__restrict__ sidx, const float *__restrict__ W,
                                                       const float *__restrict__ bias, float *__restrict__ out,
                                                       int logn) {
  __shared__ float sW[COUT * CIN * 27], sb[COUT];
  for (int i = threadIdx.x; i < COUT * CIN * 27; i += blockDim.x) sW[i] = W[i];
  if (threadIdx.x < COUT) sb[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const int n = 1 << logn, h = n >> 1, logh = logn - 1;
  const long nin = 1L << (3 * logn), nout = 1L << (3 * logh);
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nout) return;
  const int s = blockIdx.y;
  const float *src = in + (long)(sidx ? sidx[s] : s) * in_stride;
  const int qx = (int)(q & (h - 1)), qy = (int)((q >> logh) & (h - 1)), qz = (int)(q >> (2 * logh));
  const int mask = n - 1;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = sb[o];
  for (int c = 0; c < CIN; ++c) {
    const float *u = src + (long)c * nin;
    for (int dz = 0; dz < 3; ++dz) {
      const int z = (2 * qz + dz - 1) & mask;
      for (int dy = 0; dy < 3; ++dy) {
        const int y = (2 * qy + dy - 1) & mask;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int x = (2 * qx + dx - 1) & mask;
          float v = u[((long)z << (2 * logn)) + ((long)y << logn) + x];
          if (RELU_IN) v = fmaxf(v, 0.0f);
          const int t = (c * 3 + dz) * 9 + dy * 3 + dx;
#pragma unroll
          for (int o = 0; o < COUT; ++o) acc[o] = fmaf(sW[o * CIN * 27 + t], v, acc[o]);
        }
      }
    }
  }
  float *dst = out + (long)s * COUT * nout;
#pragma unroll
  for (int o = 0; o < COUT; ++o) dst[(long)o * nout + q] = acc[o];
}

// FiLM scale and shift of sample s: sa[c] = 1 + Fa[c] . phi + fa[c], sc[c] = Fc[c] . phi + fc[c]
__device__ __forceinline__ void film_coefs(const float *P, const Offs &of, const float *phi, float *sa, float *sc) {
  for (int c = threadIdx.x; c < C2; c += blockDim.x) {
    float a = 1.0f + P[of.fa + c], b = P[of.fc + c];
    for (int j = 0; j < 6; ++j) {
      a = fmaf(P[of.Fa + c * 6 + j], phi[j], a);
      b = fmaf(P[of.Fc + c * 6 + j], phi[j], b);
    }
    sa[c] = a;
    sc[c] = b;
  }
}

// z = sa relu(a2) + sc and the head h = Wh z + bh, written as the coarse complex block [s][b][comp][q].
// grid (ceil(m3 / 256), S)
__global__ void __launch_bounds__(TPB) film_head_kernel(const float *__restrict__ a2, const float *__restrict__ P,
                                                        const Offs of, const float *__restrict__ phi, int nb, long m3,
                                                        float *__restrict__ z, float2 *__restrict__ coarse) {
  __shared__ float sa[C2], sc[C2], sWh[6 * NBMAX * C2], sbh[6 * NBMAX];
  const int s = blockIdx.y;
  film_coefs(P, of, phi + 6 * s, sa, sc);
  for (int i = threadIdx.x; i < 6 * nb * C2; i += blockDim.x) sWh[i] = P[of.Wh + i];
  for (int i = threadIdx.x; i < 6 * nb; i += blockDim.x) sbh[i] = P[of.bh + i];
  __syncthreads();
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m3) return;
  float zc[C2];
#pragma unroll
  for (int c = 0; c < C2; ++c) {
    zc[c] = fmaf(sa[c], fmaxf(a2[((long)s * C2 + c) * m3 + q], 0.0f), sc[c]);
    z[((long)s * C2 + c) * m3 + q] = zc[c];
  }
  for (int bc = 0; bc < 3 * nb; ++bc) {  // (band, component) pairs; channel 2 bc is re, 2 bc + 1 is im
    float re = sbh[2 * bc], im = sbh[2 * bc + 1];
#pragma unroll
    for (int c = 0; c < C2; ++c) {
      re = fmaf(sWh[(2 * bc) * C2 + c], zc[c], re);
      im = fmaf(sWh[(2 * bc + 1) * C2 + c], zc[c], im);
    }
    coarse[((long)s * 3 * nb + bc) * m3 + q] = make_float2(re, im);
  }
}

// mean of z over the coarse points per channel, then y = Wv [mean z; phi] + bv. grid (S), TPB threads
__global__ void __launch_bounds__(TPB) pool_value_kernel(const float *__restrict__ z, const float *__restrict__ P,
                                                         const Offs of, const float *__restrict__ phi, int nb, long m3,
                                                         float *__restrict__ pool, float *__restrict__ y) {
  __shared__ float red[TPB];
  __shared__ float sp[C2];
  const int s = blockIdx.x;
  for (int c = 0; c < C2; ++c) {
    float acc = 0.0f;
    for (long q = threadIdx.x; q < m3; q += blockDim.x) acc += z[((long)s * C2 + c) * m3 + q];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sp[c] = red[0] / (float)m3;
    __syncthreads();
  }
  if ((int)threadIdx.x < C2) pool[(long)s * C2 + threadIdx.x] = sp[threadIdx.x];
  if ((int)threadIdx.x < nb) {
    const int b = threadIdx.x;
    float v = P[of.bv + b];
    for (int c = 0; c < C2; ++c) v = fmaf(P[of.Wv + b * (C2 + 6) + c], sp[c], v);
    for (int j = 0; j < 6; ++j) v = fmaf(P[of.Wv + b * (C2 + 6) + C2 + j], phi[6 * s + j], v);
    y[(long)s * nb + b] = v;
  }
}

// X[s][b][comp][i] = periodic linear interpolation of the coarse block: along each axis fine point i = 4 j + r takes
// (1 - r/4) c_j + (r/4) c_{j+1}. grid (ceil(N^3 / 256), 3 nb, S)
__global__ void __launch_bounds__(TPB) upsample_kernel(const float2 *__restrict__ coarse, float2 *__restrict__ X,
                                                       int logN) {
  const int N = 1 << logN, M = N >> 2, logM = logN - 2;
  const long n = 1L << (3 * logN), m3 = 1L << (3 * logM);
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long col = (long)blockIdx.z * gridDim.y + blockIdx.y;  // (s, band, component)
  const float2 *c = coarse + col * m3;
  const int ix = (int)(i & (N - 1)), iy = (int)((i >> logN) & (N - 1)), iz = (int)(i >> (2 * logN));
  int j0[3], j1[3];
  float w1[3];
  const int id[3] = {ix, iy, iz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    j0[a] = id[a] >> 2;
    j1[a] = (j0[a] + 1) & (M - 1);
    w1[a] = 0.25f * (float)(id[a] & 3);
  }
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int jx = (t & 1) ? j1[0] : j0[0], jy = (t & 2) ? j1[1] : j0[1], jz = (t & 4) ? j1[2] : j0[2];
    const float w = ((t & 1) ? w1[0] : 1.0f - w1[0]) * ((t & 2) ? w1[1] : 1.0f - w1[1]) *
                    ((t & 4) ? w1[2] : 1.0f - w1[2]);
    const float2 v = c[((long)jz << (2 * logM)) + ((long)jy << logM) + jx];
    acc.x = fmaf(w, v.x, acc.x);
    acc.y = fmaf(w, v.y, acc.y);
  }
  X[col * n + i] = acc;
}

// ------------------------------------------------------------------------------------------------------ loss
// Per sample (one block of NBMAX^2 threads, thread t owning entry (t / nb, t % nb) of the nb x nb matrices in shared
// memory): G = X^H X and B = X^H V (complex128, row-major), T = G^{-1} B B^H,
// loss = nb - Re tr T + w sum_b (y_b - log lambda_b)^2; the coefficients of the gradient dX = X Cx + V Cv,
// Cx = (2/S) G^{-1} B B^H G^{-1}, Cv = -(2/S) B^H G^{-1}, and dy = (2 w / S)(y - log lambda) (means over the S
// samples). G is Hermitian positive definite for a block of full rank; its inverse comes from Gauss-Jordan
// elimination without pivoting in FP64 (every pivot is real and positive); a non-positive pivot marks the sample
// (loss = NaN, zero gradient). grid (S), NBMAX^2 threads
__global__ void __launch_bounds__(NBMAX * NBMAX) loss_kernel(const double2 *__restrict__ G,
                                                             const double2 *__restrict__ B,
                                                             const float *__restrict__ y,
                                                             const double *__restrict__ lam, float wv, int nb, int S,
                                                             double *__restrict__ loss, double2 *__restrict__ Cx,
                                                             double2 *__restrict__ Cv, float *__restrict__ dy) {
  __shared__ double2 A[NBMAX][NBMAX + 1], Gi[NBMAX][NBMAX + 1], Bs[NBMAX][NBMAX + 1], BB[NBMAX][NBMAX + 1],
      Tm[NBMAX][NBMAX + 1];
  __shared__ int bad;
  const int s = blockIdx.x, t = threadIdx.x;
  const bool own = t < nb * nb;
  const int i = own ? t / nb : 0, j = own ? t % nb : 0;
  if (t == 0) bad = 0;
  if (own) {
    A[i][j] = G[(long)s * nb * nb + t];
    Bs[i][j] = B[(long)s * nb * nb + t];
    Gi[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    const double piv = A[k][k].x;
    if (!(piv > 0.0)) {  // uniform across the block: every thread reads the same pivot
      if (t == 0) bad = 1;
      break;
    }
    const double ip = 1.0 / piv;
    double2 f = make_double2(0.0, 0.0), ak = f, gk = f;
    if (own) {
      f = A[i][k];
      ak = cscale(A[k][j], ip);
      gk = cscale(Gi[k][j], ip);
    }
    __syncthreads();
    if (own) {
      if (i == k) {
        A[i][j] = ak;
        Gi[i][j] = gk;
      } else {
        A[i][j] = csub(A[i][j], cmul(f, ak));
        Gi[i][j] = csub(Gi[i][j], cmul(f, gk));
      }
    }
    __syncthreads();
  }
  __syncthreads();
  double2 *cx = Cx + (long)s * nb * nb, *cv = Cv + (long)s * nb * nb;
  if (bad) {
    if (own) cx[t] = cv[t] = make_double2(0.0, 0.0);
    if (t < nb) dy[(long)s * nb + t] = 0.0f;
    if (t == 0) loss[s] = nan("");
    return;
  }
  if (own) {  // BB = B B^H
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < nb; ++l) acc = cadd(acc, cmulc(Bs[j][l], Bs[i][l]));  // B_il conj(B_jl)
    BB[i][j] = acc;
  }
  __syncthreads();
  if (own) {  // T = Gi BB
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < nb; ++l) acc = cadd(acc, cmul(Gi[i][l], BB[l][j]));
    Tm[i][j] = acc;
  }
  __syncthreads();
  const double inv_s = 1.0 / S;
  if (own) {  // Cx = (2/S) T Gi, Cv = -(2/S) B^H Gi
    double2 ax = make_double2(0.0, 0.0), av = ax;
    for (int l = 0; l < nb; ++l) {
      ax = cadd(ax, cmul(Tm[i][l], Gi[l][j]));
      av = cadd(av, cmulc(Bs[l][i], Gi[l][j]));  // conj(B_li) Gi_lj
    }
    cx[t] = cscale(ax, 2.0 * inv_s);
    cv[t] = cscale(av, -2.0 * inv_s);
  }
  if (t < nb) {
    const double r = (double)y[(long)s * nb + t] - log(lam[(long)s * nb + t]);
    dy[(long)s * nb + t] = (float)(2.0 * wv * r * inv_s);
  }
  if (t == 0) {
    double tr = 0.0, vl = 0.0;
    for (int b = 0; b < nb; ++b) {
      tr += Tm[b][b].x;
      const double r = (double)y[(long)s * nb + b] - log(lam[(long)s * nb + b]);
      vl += r * r;
    }
    loss[s] = nb - tr + wv * vl;
  }
}

// ---------------------------------------------------------------------------------------------------- backward
// The transpose of upsample_kernel: coarse point j gathers the fine points i = 4 j + t, t = -3..3 per axis (periodic)
// with weights (1 - |t|/4). grid (ceil(m3 / 256), 3 nb, S)
__global__ void __launch_bounds__(TPB) upsample_bwd_kernel(const float2 *__restrict__ dX, float2 *__restrict__ dc,
                                                           int logN) {
  const int N = 1 << logN, logM = logN - 2, M = N >> 2;
  const long n = 1L << (3 * logN), m3 = 1L << (3 * logM);
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m3) return;
  const long col = (long)blockIdx.z * gridDim.y + blockIdx.y;
  const float2 *d = dX + col * n;
  const int jx = (int)(j & (M - 1)), jy = (int)((j >> logM) & (M - 1)), jz = (int)(j >> (2 * logM));
  const int mask = N - 1;
  float2 acc = make_float2(0.0f, 0.0f);
  for (int tz = -3; tz <= 3; ++tz) {
    const float wz = 1.0f - 0.25f * (float)abs(tz);
    const long zo = (long)((4 * jz + tz) & mask) << (2 * logN);
    for (int ty = -3; ty <= 3; ++ty) {
      const float wzy = wz * (1.0f - 0.25f * (float)abs(ty));
      const long yo = zo + ((long)((4 * jy + ty) & mask) << logN);
#pragma unroll
      for (int tx = -3; tx <= 3; ++tx) {
        const float w = wzy * (1.0f - 0.25f * (float)abs(tx));
        const float2 v = d[yo + ((4 * jx + tx) & mask)];
        acc.x = fmaf(w, v.x, acc.x);
        acc.y = fmaf(w, v.y, acc.y);
      }
    }
  }
  dc[col * m3 + j] = acc;
}

// dz = Wh^T dh + (Wv^T dy)[:C2] / m3 and da2 = sa dz where a2 > 0 (ReLU), per coarse point. grid (ceil(m3 / 256), S)
__global__ void __launch_bounds__(TPB) head_bwd_kernel(const float2 *__restrict__ dc, const float *__restrict__ a2,
                                                       const float *__restrict__ P, const Offs of,
                                                       const float *__restrict__ phi, const float *__restrict__ dy,
                                                       int nb, long m3, float *__restrict__ dz,
                                                       float *__restrict__ da2) {
  __shared__ float sa[C2], sc[C2], sWh[6 * NBMAX * C2], sdp[C2];
  const int s = blockIdx.y;
  film_coefs(P, of, phi + 6 * s, sa, sc);
  for (int i = threadIdx.x; i < 6 * nb * C2; i += blockDim.x) sWh[i] = P[of.Wh + i];
  for (int c = threadIdx.x; c < C2; c += blockDim.x) {
    float v = 0.0f;
    for (int b = 0; b < nb; ++b) v = fmaf(P[of.Wv + b * (C2 + 6) + c], dy[(long)s * nb + b], v);
    sdp[c] = v / (float)m3;
  }
  __syncthreads();
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m3) return;
  float acc[C2];
#pragma unroll
  for (int c = 0; c < C2; ++c) acc[c] = sdp[c];
  for (int bc = 0; bc < 3 * nb; ++bc) {
    const float2 d = dc[((long)s * 3 * nb + bc) * m3 + q];
#pragma unroll
    for (int c = 0; c < C2; ++c) acc[c] = fmaf(sWh[(2 * bc) * C2 + c], d.x, fmaf(sWh[(2 * bc + 1) * C2 + c], d.y, acc[c]));
  }
#pragma unroll
  for (int c = 0; c < C2; ++c) {
    const long at = ((long)s * C2 + c) * m3 + q;
    dz[at] = acc[c];
    da2[at] = a2[at] > 0.0f ? sa[c] * acc[c] : 0.0f;
  }
}

// block-wide sums of K values per thread into red[K][TPB]; thread 0 gets the totals in red[k][0]
template <int K> __device__ __forceinline__ void block_sum(float (*red)[TPB], const float *v) {
#pragma unroll
  for (int k = 0; k < K; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < K; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
}

// dWh[o][c] = sum_{s,q} dh[s][o][q] z[s][c][q], dbh[o] = sum dh (dh: channel o = 2 bc + ri of the coarse gradient).
// grid (6 nb), TPB threads
__global__ void __launch_bounds__(TPB) head_grad_kernel(const float2 *__restrict__ dc, const float *__restrict__ z,
                                                        int nb, int S, long m3, float *__restrict__ gWh,
                                                        float *__restrict__ gbh) {
  __shared__ float red[C2 + 1][TPB];
  const int o = blockIdx.x, bc = o >> 1, ri = o & 1;
  float acc[C2 + 1];
#pragma unroll
  for (int c = 0; c <= C2; ++c) acc[c] = 0.0f;
  const long tot = (long)S * m3;
  for (long t = threadIdx.x; t < tot; t += blockDim.x) {
    const int s = (int)(t / m3);
    const long q = t - (long)s * m3;
    const float2 d2 = dc[((long)s * 3 * nb + bc) * m3 + q];
    const float d = ri ? d2.y : d2.x;
#pragma unroll
    for (int c = 0; c < C2; ++c) acc[c] = fmaf(d, z[((long)s * C2 + c) * m3 + q], acc[c]);
    acc[C2] += d;
  }
  block_sum<C2 + 1>(red, acc);
  if (threadIdx.x == 0) {
    for (int c = 0; c < C2; ++c) gWh[o * C2 + c] = red[c][0];
    gbh[o] = red[C2][0];
  }
}

// per sample and channel: dsa = sum_q dz relu(a2), dsc = sum_q dz. grid (C2, S), TPB threads
__global__ void __launch_bounds__(TPB) film_grad_kernel(const float *__restrict__ dz, const float *__restrict__ a2,
                                                        long m3, float *__restrict__ dsa, float *__restrict__ dsc) {
  __shared__ float red[2][TPB];
  const int c = blockIdx.x, s = blockIdx.y;
  const long base = ((long)s * C2 + c) * m3;
  float acc[2] = {0.0f, 0.0f};
  for (long q = threadIdx.x; q < m3; q += blockDim.x) {
    const float d = dz[base + q];
    acc[0] = fmaf(d, fmaxf(a2[base + q], 0.0f), acc[0]);
    acc[1] += d;
  }
  block_sum<2>(red, acc);
  if (threadIdx.x == 0) {
    dsa[(long)s * C2 + c] = red[0][0];
    dsc[(long)s * C2 + c] = red[1][0];
  }
}

// gradients of FiLM and of the value head, summed over the samples (one block)
__global__ void small_grads_kernel(const float *__restrict__ dsa, const float *__restrict__ dsc,
                                   const float *__restrict__ phi, const float *__restrict__ pool,
                                   const float *__restrict__ dy, int nb, int S, const Offs of, float *__restrict__ g) {
  for (int e = threadIdx.x; e < C2 * 7; e += blockDim.x) {  // (c, j) with j = 6: the bias
    const int c = e / 7, j = e % 7;
    float a = 0.0f, b = 0.0f;
    for (int s = 0; s < S; ++s) {
      const float f = j < 6 ? phi[6 * s + j] : 1.0f;
      a = fmaf(dsa[(long)s * C2 + c], f, a);
      b = fmaf(dsc[(long)s * C2 + c], f, b);
    }
    if (j < 6) {
      g[of.Fa + c * 6 + j] = a;
      g[of.Fc + c * 6 + j] = b;
    } else {
      g[of.fa + c] = a;
      g[of.fc + c] = b;
    }
  }
  for (int e = threadIdx.x; e < nb * (C2 + 7); e += blockDim.x) {  // (b, f) with f = C2 + 6: the bias
    const int b = e / (C2 + 7), f = e % (C2 + 7);
    float a = 0.0f;
    for (int s = 0; s < S; ++s) {
      const float x = f < C2 ? pool[(long)s * C2 + f] : (f < C2 + 6 ? phi[6 * s + f - C2] : 1.0f);
      a = fmaf(dy[(long)s * nb + b], x, a);
    }
    if (f < C2 + 6) g[of.Wv + b * (C2 + 6) + f] = a;
    else g[of.bv + b] = a;
  }
}

// dW[o][c][t] = sum_{s,q} dout[s][o][q] in[s][c][2q + d - 1], db[o] = sum dout (written by the c = 0 block).
// grid (COUT, CIN), TPB threads
template <int CIN, int COUT, bool RELU_IN>
__global__ void __launch_bounds__(TPB) conv_wgrad_kernel(const float *__restrict__ dout, const float *__restrict__ in,
                                                         long in_stride, const int *__restrict__ sidx, int S, int logn,
                                                         float *__restrict__ gW, float *__restrict__ gb) {
  __shared__ float red[28][TPB];
  const int o = blockIdx.x, c = blockIdx.y;
  const int n = 1 << logn, h = n >> 1, logh = logn - 1, mask = n - 1;
  const long nin = 1L << (3 * logn), nout = 1L << (3 * logh);
  float acc[28];
#pragma unroll
  for (int t = 0; t < 28; ++t) acc[t] = 0.0f;
  const long tot = (long)S * nout;
  for (long e = threadIdx.x; e < tot; e += blockDim.x) {
    const int s = (int)(e / nout);
    const long q = e - (long)s * nout;
    const float d = dout[((long)s * COUT + o) * nout + q];
    const float *u = in + (long)(sidx ? sidx[s] : s) * in_stride + (long)c * nin;
    const int qx = (int)(q & (h - 1)), qy = (int)((q >> logh) & (h - 1)), qz = (int)(q >> (2 * logh));
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
      const int zz = (2 * qz + dz - 1) & mask;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const int yy = (2 * qy + dy - 1) & mask;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int xx = (2 * qx + dx - 1) & mask;
          float v = u[((long)zz << (2 * logn)) + ((long)yy << logn) + xx];
          if (RELU_IN) v = fmaxf(v, 0.0f);
          acc[dz * 9 + dy * 3 + dx] = fmaf(d, v, acc[dz * 9 + dy * 3 + dx]);
        }
      }
    }
    acc[27] += d;
  }
  block_sum<28>(red, acc);
  if (threadIdx.x == 0) {
    for (int t = 0; t < 27; ++t) gW[(o * CIN + c) * 27 + t] = red[t][0];
    if (c == 0) gb[o] = red[27][0];
  }
}

// The transposed convolution as a gather, with the ReLU mask of its input: din[s][c][p] = [a_in > 0]
// sum_{o,d} W[o][c][d] dout[s][o][q] over the taps with 2q + d - 1 = p (mod n) per axis (an even p has the centre
// tap only, an odd p the two outer ones). grid (ceil(nin / 256), S)
template <int CIN, int COUT>
__global__ void __launch_bounds__(TPB) conv_dgrad_kernel(const float *__restrict__ dout, const float *__restrict__ W,
                                                         const float *__restrict__ a_in, int logn,
                                                         float *__restrict__ din) {
  __shared__ float sW[COUT * CIN * 27];
  for (int i = threadIdx.x; i < COUT * CIN * 27; i += blockDim.x) sW[i] = W[i];
  __syncthreads();
  const int n = 1 << logn, logh = logn - 1, mask = n - 1;
  const long nin = 1L << (3 * logn), nout = 1L << (3 * logh);
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nin) return;
  const int s = blockIdx.y;
  const int pc[3] = {(int)(p & mask), (int)((p >> logn) & mask), (int)(p >> (2 * logn))};
  // per axis: the taps d (0..2) with p - d + 1 even and their output index q = ((p - d + 1) mod n) / 2
  int nt[3], td[3][2], tq[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    nt[a] = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int r = (pc[a] - d + 1 + n) & mask;
      if ((r & 1) == 0) {
        td[a][nt[a]] = d;
        tq[a][nt[a]] = r >> 1;
        ++nt[a];
      }
    }
  }
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.0f;
  for (int iz = 0; iz < nt[2]; ++iz)
    for (int iy = 0; iy < nt[1]; ++iy)
      for (int ix = 0; ix < nt[0]; ++ix) {
        const int t = td[2][iz] * 9 + td[1][iy] * 3 + td[0][ix];
        const long q = ((long)tq[2][iz] << (2 * logh)) + ((long)tq[1][iy] << logh) + tq[0][ix];
        for (int o = 0; o < COUT; ++o) {
          const float d = dout[((long)s * COUT + o) * nout + q];
#pragma unroll
          for (int c = 0; c < CIN; ++c) acc[c] = fmaf(sW[(o * CIN + c) * 27 + t], d, acc[c]);
        }
      }
#pragma unroll
  for (int c = 0; c < CIN; ++c) {
    const long at = ((long)s * CIN + c) * nin + p;
    din[at] = a_in[at] > 0.0f ? acc[c] : 0.0f;
  }
}

// Adam (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr m^ / (sqrt(v^) + eps) with the bias
// corrections m^ = m / (1 - b1^t), v^ = v / (1 - b2^t) passed in as c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
__global__ void adam_kernel(long P, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

}  // namespace ws
}  // namespace pc

using namespace pc;
using namespace pc::ws;

namespace {

int check_dims(int N, int nb, int S) {
  PC_REQUIRE(is_pow2(N) && N >= 16 && N <= 256, "warm start: N must be a power of two in [16, 256], got %d", N);
  PC_REQUIRE(nb >= 1 && nb <= NBMAX, "warm start: nb must be in [1, %d], got %d", NBMAX, nb);
  PC_REQUIRE(S >= 1 && S <= 65535, "warm start: S must be in [1, 65535], got %d", S);
  return PC_OK;
}

char *wp(void *work, size_t off) { return static_cast<char *>(work) + off; }

// every sample's structure index must address one of the nstruct M0 grids (read back from the device: S ints)
int check_sidx(const int *sidx, int S, int nstruct, cudaStream_t st) {
  std::vector<int> h(S);
  PC_CK(cudaMemcpyAsync(h.data(), sidx, sizeof(int) * S, cudaMemcpyDeviceToHost, st));
  PC_CK(cudaStreamSynchronize(st));
  for (int s = 0; s < S; ++s)
    PC_REQUIRE(h[s] >= 0 && h[s] < nstruct, "warm start: sidx[%d] = %d is outside [0, %d)", s, h[s], nstruct);
  return PC_OK;
}

}  // namespace

extern "C" long pc_ws_param_count(int nb) {
  if (nb < 1 || nb > NBMAX) return -1;
  return offsets(nb).total;
}

extern "C" size_t pc_ws_work_bytes(int N, int nb, int S) {
  if (!is_pow2(N) || N < 16 || N > 256 || nb < 1 || nb > NBMAX || S < 1) return 0;
  return work_layout(N, nb, S).total;
}

extern "C" int pc_ws_forward(int N, int nb, int S, const float *params, const float *m0, int nstruct,
                             const int *sidx, const double *kpts, void *X, float *y, void *work, void *stream) {
  int rc = check_dims(N, nb, S);
  if (rc) return rc;
  PC_REQUIRE(params && m0 && sidx && kpts && X && y && work, "pc_ws_forward: null argument");
  PC_REQUIRE(nstruct >= 1, "pc_ws_forward: nstruct must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  rc = check_sidx(sidx, S, nstruct, st);
  if (rc) return rc;
  const Offs of = offsets(nb);
  const Work w = work_layout(N, nb, S);
  const int logN = ilog2(N);
  const long n = (long)N * N * N, n1 = n / 8, m3 = n / 64;
  std::vector<float> phi(6 * (size_t)S);
  for (int s = 0; s < S; ++s)
    for (int a = 0; a < 3; ++a) {
      phi[6 * s + a] = (float)std::sin(kpts[3 * s + a]);
      phi[6 * s + 3 + a] = (float)std::cos(kpts[3 * s + a]);
    }
  float *dphi = reinterpret_cast<float *>(wp(work, w.phi));
  PC_CK(cudaMemcpyAsync(dphi, phi.data(), sizeof(float) * phi.size(), cudaMemcpyHostToDevice, st));
  float *a1 = reinterpret_cast<float *>(wp(work, w.a1)), *a2 = reinterpret_cast<float *>(wp(work, w.a2));
  float *z = reinterpret_cast<float *>(wp(work, w.z)), *pool = reinterpret_cast<float *>(wp(work, w.pool));
  float2 *coarse = reinterpret_cast<float2 *>(wp(work, w.coarse));
  conv_fwd_kernel<3, C1, false><<<dim3((unsigned)((n1 + TPB - 1) / TPB), S), TPB, 0, st>>>(
      m0, 3 * n, sidx, params + of.W1, params + of.b1, a1, logN);
  PC_CK_LAUNCH();
  conv_fwd_kernel<C1, C2, true><<<dim3((unsigned)((m3 + TPB - 1) / TPB), S), TPB, 0, st>>>(
      a1, C1 * n1, nullptr, params + of.W2, params + of.b2, a2, logN - 1);
  PC_CK_LAUNCH();
  film_head_kernel<<<dim3((unsigned)((m3 + TPB - 1) / TPB), S), TPB, 0, st>>>(a2, params, of, dphi, nb, m3, z, coarse);
  PC_CK_LAUNCH();
  pool_value_kernel<<<S, TPB, 0, st>>>(z, params, of, dphi, nb, m3, pool, y);
  PC_CK_LAUNCH();
  upsample_kernel<<<dim3((unsigned)((n + TPB - 1) / TPB), 3 * nb, S), TPB, 0, st>>>(coarse, static_cast<float2 *>(X),
                                                                                   logN);
  PC_CK_LAUNCH();
  PC_CK(cudaStreamSynchronize(st));  // the host copy of phi goes out of scope
  return PC_OK;
}

extern "C" int pc_ws_backward(int N, int nb, int S, const float *params, const float *m0, int nstruct,
                              const int *sidx, const void *X, const float *y, const void *V, const double *lam,
                              float w_val, float *grad, double *loss, void *work, void *stream) {
  int rc = check_dims(N, nb, S);
  if (rc) return rc;
  PC_REQUIRE(params && m0 && sidx && X && y && V && lam && grad && loss && work, "pc_ws_backward: null argument");
  PC_REQUIRE(w_val >= 0.0f, "pc_ws_backward: w_val must be >= 0");
  PC_REQUIRE(nstruct >= 1, "pc_ws_backward: nstruct must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  rc = check_sidx(sidx, S, nstruct, st);
  if (rc) return rc;
  const Offs of = offsets(nb);
  const Work w = work_layout(N, nb, S);
  const int logN = ilog2(N);
  const long n = (long)N * N * N, n1 = n / 8, m3 = n / 64, L = 3 * n;
  const float *dphi = reinterpret_cast<const float *>(wp(work, w.phi));
  float *a1 = reinterpret_cast<float *>(wp(work, w.a1)), *a2 = reinterpret_cast<float *>(wp(work, w.a2));
  float *z = reinterpret_cast<float *>(wp(work, w.z)), *pool = reinterpret_cast<float *>(wp(work, w.pool));
  float *dy = reinterpret_cast<float *>(wp(work, w.dy));
  double2 *G = reinterpret_cast<double2 *>(wp(work, w.G)), *B = reinterpret_cast<double2 *>(wp(work, w.B));
  double2 *Cx = reinterpret_cast<double2 *>(wp(work, w.Cx)), *Cv = reinterpret_cast<double2 *>(wp(work, w.Cv));
  float2 *dX = reinterpret_cast<float2 *>(wp(work, w.dX)), *dc = reinterpret_cast<float2 *>(wp(work, w.dcoarse));
  float *dz = reinterpret_cast<float *>(wp(work, w.dz)), *da2 = reinterpret_cast<float *>(wp(work, w.da2));
  float *da1 = reinterpret_cast<float *>(wp(work, w.da1));
  float *dsa = reinterpret_cast<float *>(wp(work, w.dsa)), *dsc = reinterpret_cast<float *>(wp(work, w.dsc));
  double *dloss = reinterpret_cast<double *>(wp(work, w.loss));
  void *gscr = wp(work, w.gram);
  const size_t gbytes = std::max<size_t>(16, gram_scratch_bytes(S, L, nb, nb));
  const long sx = (long)nb * L;
  // subspace loss and its gradient in X
  rc = launch_gram(S, L, nb, nb, PC_C64, X, sx, X, sx, G, gscr, gbytes, st, nullptr);
  if (rc) return rc;
  rc = launch_gram(S, L, nb, nb, PC_C64, X, sx, V, sx, B, gscr, gbytes, st, nullptr);
  if (rc) return rc;
  loss_kernel<<<S, NBMAX * NBMAX, 0, st>>>(G, B, y, lam, w_val, nb, S, dloss, Cx, Cv, dy);
  PC_CK_LAUNCH();
  rc = launch_block_update(S, L, nb, nb, PC_C64, X, sx, Cx, (long)nb * nb, dX, sx, st, nullptr);
  if (rc) return rc;
  rc = launch_block_update(S, L, nb, nb, PC_C64, V, sx, Cv, (long)nb * nb, dX, sx, st, nullptr, dX, sx);
  if (rc) return rc;
  // back through the upsampling, the head, FiLM and the value head
  upsample_bwd_kernel<<<dim3((unsigned)((m3 + TPB - 1) / TPB), 3 * nb, S), TPB, 0, st>>>(dX, dc, logN);
  PC_CK_LAUNCH();
  head_bwd_kernel<<<dim3((unsigned)((m3 + TPB - 1) / TPB), S), TPB, 0, st>>>(dc, a2, params, of, dphi, dy, nb, m3, dz,
                                                                            da2);
  PC_CK_LAUNCH();
  head_grad_kernel<<<6 * nb, TPB, 0, st>>>(dc, z, nb, S, m3, grad + of.Wh, grad + of.bh);
  PC_CK_LAUNCH();
  film_grad_kernel<<<dim3(C2, S), TPB, 0, st>>>(dz, a2, m3, dsa, dsc);
  PC_CK_LAUNCH();
  small_grads_kernel<<<1, TPB, 0, st>>>(dsa, dsc, dphi, pool, dy, nb, S, of, grad);
  PC_CK_LAUNCH();
  // back through the encoder
  conv_wgrad_kernel<C1, C2, true><<<dim3(C2, C1), TPB, 0, st>>>(da2, a1, C1 * n1, nullptr, S, logN - 1,
                                                                 grad + of.W2, grad + of.b2);
  PC_CK_LAUNCH();
  conv_dgrad_kernel<C1, C2><<<dim3((unsigned)((n1 + TPB - 1) / TPB), S), TPB, 0, st>>>(da2, params + of.W2, a1,
                                                                                       logN - 1, da1);
  PC_CK_LAUNCH();
  conv_wgrad_kernel<3, C1, false><<<dim3(C1, 3), TPB, 0, st>>>(da1, m0, 3 * n, sidx, S, logN, grad + of.W1,
                                                               grad + of.b1);
  PC_CK_LAUNCH();
  PC_CK(cudaMemcpyAsync(loss, dloss, sizeof(double) * S, cudaMemcpyDeviceToDevice, st));
  return PC_OK;
}

extern "C" int pc_ws_adam(long P, float *params, const float *grad, float *m, float *v, int t, float lr, float b1,
                          float b2, float eps, void *stream) {
  PC_REQUIRE(params && grad && m && v, "pc_ws_adam: null argument");
  PC_REQUIRE(P >= 0 && t >= 1, "pc_ws_adam: need P >= 0 and step t >= 1");
  PC_REQUIRE(lr > 0.0f && b1 >= 0.0f && b1 < 1.0f && b2 >= 0.0f && b2 < 1.0f && eps > 0.0f, "pc_ws_adam: bad hyperparameters");
  if (P == 0) return PC_OK;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, t))), c2 = (float)(1.0 / (1.0 - std::pow((double)b2, t)));
  adam_kernel<<<(unsigned)((P + TPB - 1) / TPB), TPB, 0, (cudaStream_t)stream>>>(P, params, grad, m, v, lr, b1, b2, eps,
                                                                               c1, c2);
  PC_CK_LAUNCH();
  return PC_OK;
}
