// Complex64 FFT preconditioner W = P^{-1} R (Section 5.2, Algorithm 5.1, with the 3x3 mode symbol of
// eq. penalised_marix) for N = 8 .. 128: three passes over the block, each one HBM read and one HBM write.
//   1. forward transforms along x and y of one (component, z) plane held in shared memory;
//   2. along z, all three components of U consecutive (x, y) columns: forward transform, the exact inverse of the
//      mode's 3x3 symbol sigma I + (gamma - 1) conj(d) d^T times 1/N^3, inverse transform;
//   3. inverse transforms along y and x of each plane.
// Every line transform of length N = N1 N2 (N1 <= N2 <= 16, both powers of two) is split in two (Cooley-Tukey with
// n = n1 + N1 n2, k = k2 + N2 k1): N1 threads each take one DFT of length N2 over the stride-N1 elements of the
// line in registers, multiply by the twiddles W_N^(n1 k2), exchange through shared memory, and take N2/N1 DFTs of
// length N1. Inputs and outputs are in natural order, so the symbol is applied at the natural mode indices. The
// small DFTs are radix-2 decimation in time on registers with the constant roots of unity of order 16.
//
// Shared-memory layouts are chosen so that every warp access touches each bank pair at most twice (two wavefronts
// for 32 eight-byte accesses, the minimum): the x pass of the plane kernel runs with consecutive threads on the
// N1 pieces of a line (coalesced global loads of N1 consecutive elements per row), its exchange rows padded to
// N + N1 entries with the pieces at stride N2 + 1; the y pass runs with consecutive threads on consecutive columns
// (conflict-free row segments in shared memory and coalesced 256-byte stores to global memory); the z pass has
// consecutive threads on consecutive columns as well.
#include <cmath>

#include "pc_internal.cuh"

namespace pc {

namespace {

constexpr int clog2(int n) { return n <= 1 ? 0 : 1 + clog2(n / 2); }
constexpr int cbrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
// cos(2 pi e / 16) for e = 0 .. 15
__host__ __device__ constexpr float cos16(int e) {
  switch (e & 15) {
    case 0: return 1.0f;
    case 1: case 15: return 0.92387953251128676f;
    case 2: case 14: return 0.70710678118654752f;
    case 3: case 13: return 0.38268343236508977f;
    case 4: case 12: return 0.0f;
    case 5: case 11: return -0.38268343236508977f;
    case 6: case 10: return -0.70710678118654752f;
    case 7: case 9: return -0.92387953251128676f;
    default: return -1.0f;
  }
}

// x * exp(-2 pi i e / 16) (forward) or x * exp(+2 pi i e / 16) (inverse); e is a compile-time constant after unrolling
template <bool INV> __device__ __forceinline__ float2 rot16(float2 x, int e) {
  e &= 15;
  if (e == 0) return x;
  if (e == 8) return make_float2(-x.x, -x.y);
  if (e == 4) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
  if (e == 12) return INV ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
  const float c = cos16(e), s = cos16(e - 4);  // sin(t) = cos(t - pi / 2)
  return INV ? make_float2(x.x * c - x.y * s, x.x * s + x.y * c) : make_float2(x.x * c + x.y * s, x.y * c - x.x * s);
}

// In-register DFT of length R <= 16 (natural order in and out): radix-2 decimation in time after the bit-reversal
// permutation (a renaming of registers).
template <int R, bool INV> __device__ __forceinline__ void dft(float2 *v) {
  if constexpr (R > 1) {
    constexpr int LOG = clog2(R);
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[cbrev(i, LOG)];
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
      for (int blk = 0; blk < R; blk += len) {
#pragma unroll
        for (int j = 0; j < len / 2; ++j) {
          const float2 a = t[blk + j];
          const float2 b = rot16<INV>(t[blk + j + len / 2], j * (16 / len));
          t[blk + j] = make_float2(a.x + b.x, a.y + b.y);
          t[blk + j + len / 2] = make_float2(a.x - b.x, a.y - b.y);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
  }
}

// x * w (forward) or x * conj(w) (inverse)
template <bool INV> __device__ __forceinline__ float2 twmul(float2 x, float2 w) {
  return INV ? make_float2(x.x * w.x + x.y * w.y, x.y * w.x - x.x * w.y)
             : make_float2(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
}

// Split of a length-N transform: N1 <= N2 <= 16.
template <int N> struct Split {
  static constexpr int N1 = N <= 8 ? 2 : (N <= 32 ? 4 : (N <= 128 ? 8 : 16));
  static constexpr int N2 = N / N1;
  static_assert(N1 * N2 == N && N1 <= N2 && N2 <= 16, "unsupported length");
};

// planes per CTA (about 512 threads; P divides the 3N planes of a field) and whether the plane kernel's exchange
// shares the plane buffer (for N = 128 two N x (N + N1) buffers would not fit in shared memory)
template <int N> struct PlaneCfg {
  static constexpr int N1 = Split<N>::N1;
  static constexpr int P0 = (N * N1 >= 512) ? 1 : 512 / (N * N1);
  static constexpr int P = P0 < N ? P0 : N;
  static constexpr int LD = N + N1;  // row stride (elements) of the plane and exchange buffers
  static constexpr bool SINGLE = N >= 128;
  static constexpr int THREADS = P * N * N1;
  static constexpr size_t smem() {
    return sizeof(float2) * ((size_t)(SINGLE ? 1 : 2) * P * N * LD + N);
  }
};

// twiddle table W_N^t = exp(-2 pi i t / N), t < N, from the context's table of the first N / 2
__device__ __forceinline__ void load_twiddles(float2 *s_tw, const float2 *tw, int N) {
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
    const float2 w = tw[t];
    s_tw[t] = w;
    s_tw[t + N / 2] = make_float2(-w.x, -w.y);
  }
}

// Forward (x then y) or inverse (y then x) transforms of P planes (component, z) per CTA. grid (3N / P, m, nb).
template <int N, bool FWD>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS) fft_plane_kernel(const float2 *__restrict__ in, long si,
                                                                         float2 *__restrict__ out, long so,
                                                                         const float2 *__restrict__ tw,
                                                                         const int *__restrict__ act) {
  using CF = PlaneCfg<N>;
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, P = CF::P, LD = CF::LD, Q = N2 / N1;
  constexpr bool INV = !FWD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *s_tw = reinterpret_cast<float2 *>(smem_raw);
  float2 *A = s_tw + N;                                  // planes [P N rows][LD]
  float2 *E = CF::SINGLE ? A : A + (size_t)P * N * LD;   // exchange [P N rows][LD]
  const long n = (long)N * N * N;
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const long off = (long)blockIdx.y * 3 * n + (long)blockIdx.x * P * N * N;
  const float2 *src = in + (long)b * si + off;
  float2 *dst = out + (long)b * so + off;
  load_twiddles(s_tw, tw, N);
  float2 v[N2];

  // ---- first pass: along x (forward) or y (inverse) on lines owned by N1 consecutive threads
  // forward: line = row (plane, y), loads of the row's elements x = n1 + N1 n2 straight from global memory
  // inverse: line = column (plane, x): consecutive threads on consecutive columns
  const int tid = threadIdx.x;
  if (FWD) {
    const int n1 = tid % N1, row = tid / N1;
#pragma unroll
    for (int j = 0; j < N2; ++j) v[j] = src[(long)row * N + n1 + N1 * j];
    __syncthreads();  // twiddle table
    dft<N2, INV>(v);
#pragma unroll
    for (int j = 1; j < N2; ++j) v[j] = twmul<INV>(v[j], s_tw[n1 * j]);
#pragma unroll
    for (int j = 0; j < N2; ++j) E[row * LD + n1 * (N2 + 1) + j] = v[j];
    __syncthreads();
    const int t = n1;
    float2 u[N2];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) u[q * N1 + a] = E[row * LD + a * (N2 + 1) + t + N1 * q];
#pragma unroll
    for (int q = 0; q < Q; ++q) dft<N1, INV>(u + q * N1);
    if (CF::SINGLE) __syncthreads();  // E is A: every exchange read done before the plane is written
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) A[row * LD + t + N1 * q + N2 * a] = u[q * N1 + a];
  } else {
    const int x = tid % N, r = tid / N, p = r % P, m1 = r / P;
#pragma unroll
    for (int j = 0; j < N2; ++j) v[j] = src[(long)p * N * N + (long)(m1 + N1 * j) * N + x];
    __syncthreads();
    dft<N2, INV>(v);
#pragma unroll
    for (int j = 1; j < N2; ++j) v[j] = twmul<INV>(v[j], s_tw[m1 * j]);
#pragma unroll
    for (int j = 0; j < N2; ++j) E[(p * N + m1 * N2 + j) * LD + x] = v[j];
    __syncthreads();
    float2 u[N2];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) u[q * N1 + a] = E[(p * N + a * N2 + m1 + N1 * q) * LD + x];
#pragma unroll
    for (int q = 0; q < Q; ++q) dft<N1, INV>(u + q * N1);
    if (CF::SINGLE) __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) A[(p * N + m1 + N1 * q + N2 * a) * LD + x] = u[q * N1 + a];
  }
  __syncthreads();

  // ---- second pass: along y (forward) or x (inverse)
  if (FWD) {
    // line = column (plane, x), consecutive threads on consecutive columns; results stored straight to global memory
    const int x = tid % N, r = tid / N, p = r % P, m1 = r / P;
#pragma unroll
    for (int j = 0; j < N2; ++j) v[j] = A[(p * N + m1 + N1 * j) * LD + x];
    dft<N2, INV>(v);
#pragma unroll
    for (int j = 1; j < N2; ++j) v[j] = twmul<INV>(v[j], s_tw[m1 * j]);
    if (CF::SINGLE) __syncthreads();
#pragma unroll
    for (int j = 0; j < N2; ++j) E[(p * N + m1 * N2 + j) * LD + x] = v[j];
    __syncthreads();
    float2 u[N2];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) u[q * N1 + a] = E[(p * N + a * N2 + m1 + N1 * q) * LD + x];
#pragma unroll
    for (int q = 0; q < Q; ++q) dft<N1, INV>(u + q * N1);
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) dst[(long)p * N * N + (long)(m1 + N1 * q + N2 * a) * N + x] = u[q * N1 + a];
  } else {
    // line = row (plane, y), the N1 pieces on consecutive threads; stores of N1 consecutive elements per row
    const int n1 = tid % N1, row = tid / N1;
#pragma unroll
    for (int j = 0; j < N2; ++j) v[j] = A[row * LD + n1 + N1 * j];
    dft<N2, INV>(v);
#pragma unroll
    for (int j = 1; j < N2; ++j) v[j] = twmul<INV>(v[j], s_tw[n1 * j]);
    if (CF::SINGLE) __syncthreads();
#pragma unroll
    for (int j = 0; j < N2; ++j) E[row * LD + n1 * (N2 + 1) + j] = v[j];
    __syncthreads();
    const int t = n1;
    float2 u[N2];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) u[q * N1 + a] = E[row * LD + a * (N2 + 1) + t + N1 * q];
#pragma unroll
    for (int q = 0; q < Q; ++q) dft<N1, INV>(u + q * N1);
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int a = 0; a < N1; ++a) dst[(long)row * N + t + N1 * q + N2 * a] = u[q * N1 + a];
  }
}

// columns per CTA of the z pass: about 384 threads (3 U N1), U <= N^2
template <int N> struct ZCfg {
  static constexpr int N1 = Split<N>::N1;
  static constexpr int U0 = 512 / (3 * N1) >= 64 ? 64 : (512 / (3 * N1) >= 32 ? 32 : 16);
  static constexpr int U = U0 <= N * N ? U0 : N * N;
  static constexpr int THREADS = 3 * U * N1;
  static constexpr size_t smem() {
    // exchange [3][N][U], modes [3][N][U], twiddles N, symbols: x/y parts [U][3][2] and z part [3][N]
    return sizeof(float2) * (2 * (size_t)3 * N * U + N + 6 * (size_t)U + 3 * (size_t)N);
  }
};

// Along z with the symbol, for U consecutive (x, y) columns (flattened index xy = y N + x) and all 3 components.
// grid (N^2 / U, m, nb). LAT: general lattice (Section 4.2.2), d_i = sum_j (part of axis j)(m_j) from the tables
// [b][i][j][N]; otherwise d_i from the per-axis tables [b][i][N].
template <int N, bool LAT>
__global__ void __launch_bounds__(ZCfg<N>::THREADS) fft_zsym_kernel(const float2 *__restrict__ in, long si,
                                                                    float2 *__restrict__ out, long so,
                                                                    const float2 *__restrict__ tw,
                                                                    const double2 *__restrict__ sym,
                                                                    const KParam *__restrict__ kp,
                                                                    const int *__restrict__ act, int laplacian) {
  using CF = ZCfg<N>;
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, U = CF::U, Q = N2 / N1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *E = reinterpret_cast<float2 *>(smem_raw);  // [3][N][U]
  float2 *S = E + 3 * N * U;                         // [3][N][U]
  float2 *s_tw = S + 3 * N * U;                      // [N]
  float2 *dxy = s_tw + N;                            // [U][3]: x and y parts of d_i at each column
  float2 *dz = dxy + 3 * U;                          // [3][N]: z part of d_i (on the cube: d_3 itself)
  const long n = (long)N * N * N;
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int xy0 = blockIdx.x * U;
  const long base_i = (long)b * si + (long)blockIdx.y * 3 * n + xy0;
  const long base_o = (long)b * so + (long)blockIdx.y * 3 * n + xy0;
  load_twiddles(s_tw, tw, N);
  {
    const double2 *symb = sym + (long)b * (LAT ? 9 : 3) * N;
    for (int i = threadIdx.x; i < 3 * U; i += blockDim.x) {
      const int u = i / 3, c = i % 3;
      const int xx = (xy0 + u) % N, yy = (xy0 + u) / N;
      double re, im;
      if (LAT) {
        const double2 px = symb[(c * 3 + 0) * N + xx], py = symb[(c * 3 + 1) * N + yy];
        re = px.x + py.x;
        im = px.y + py.y;
      } else {
        // cube: d_1 depends on x, d_2 on y, d_3 on z only
        const double2 d = c == 0 ? symb[xx] : (c == 1 ? symb[N + yy] : make_double2(0.0, 0.0));
        re = d.x;
        im = d.y;
      }
      dxy[u * 3 + c] = make_float2((float)re, (float)im);
    }
    for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) {
      const int c = i / N, zz = i % N;
      const double2 d = LAT ? symb[(c * 3 + 2) * N + zz] : (c == 2 ? symb[2 * N + zz] : make_double2(0.0, 0.0));
      dz[i] = make_float2((float)d.x, (float)d.y);
    }
  }
  const int tid = threadIdx.x;
  const int u = tid % U, r = tid / U, n1 = r % N1, c = r / N1;
  float2 v[N2];
#pragma unroll
  for (int j = 0; j < N2; ++j) v[j] = in[base_i + (long)c * n + (long)(n1 + N1 * j) * N * N + u];
  __syncthreads();  // twiddles and symbols
  // forward along z
  dft<N2, false>(v);
#pragma unroll
  for (int j = 1; j < N2; ++j) v[j] = twmul<false>(v[j], s_tw[n1 * j]);
#pragma unroll
  for (int j = 0; j < N2; ++j) E[(c * N + n1 * N2 + j) * U + u] = v[j];
  __syncthreads();
  const int t = n1;
  float2 w[N2];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int a = 0; a < N1; ++a) w[q * N1 + a] = E[(c * N + a * N2 + t + N1 * q) * U + u];
#pragma unroll
  for (int q = 0; q < Q; ++q) dft<N1, false>(w + q * N1);
  // mode kz = k2 + N2 k1 with k2 = t + N1 q: all three components into S
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int a = 0; a < N1; ++a) S[(c * N + t + N1 * q + N2 * a) * U + u] = w[q * N1 + a];
  __syncthreads();
  // the symbol's inverse, one mode (all three components) per thread and step: consecutive threads on consecutive
  // columns, each mode's sigma, reciprocal and d^T r formed once
  {
    const float fac = kp[b].pfacf;  // (gamma - 1) / gamma
    const float scale = 1.0f / (float)n;
    for (int i = tid; i < U * N; i += CF::THREADS) {
      const int uu = i % U, kz = i / U;
      const float2 d1 = cadd(dxy[uu * 3 + 0], dz[kz]), d2 = cadd(dxy[uu * 3 + 1], dz[N + kz]);
      const float2 d3 = cadd(dxy[uu * 3 + 2], dz[2 * N + kz]);
      const float sigma = d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y + d3.x * d3.x + d3.y * d3.y;
      float2 *m = S + kz * U + uu;
      float2 r1 = m[0], r2 = m[N * U], r3 = m[2 * N * U];
      if (!(sigma > 0.f)) {
        r1 = r2 = r3 = make_float2(0.f, 0.f);
      } else {
        const float rs = __frcp_rn(sigma);
        if (!laplacian) {
          // r_c - (gamma - 1) / (gamma sigma) conj(d_c) (d^T r)
          const float2 sd = cscale(cadd(cadd(cmul(d1, r1), cmul(d2, r2)), cmul(d3, r3)), fac * rs);
          r1 = csub(r1, cmulc(d1, sd));
          r2 = csub(r2, cmulc(d2, sd));
          r3 = csub(r3, cmulc(d3, sd));
        }
        const float f = scale * rs;
        r1 = cscale(r1, f);
        r2 = cscale(r2, f);
        r3 = cscale(r3, f);
      }
      m[0] = r1;
      m[N * U] = r2;
      m[2 * N * U] = r3;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int a = 0; a < N1; ++a) w[q * N1 + a] = S[(c * N + t + N1 * q + N2 * a) * U + u];
  // inverse along z: the length-N1 DFTs first (over k1), twiddles, exchange, the length-N2 DFTs (over k2)
#pragma unroll
  for (int q = 0; q < Q; ++q) dft<N1, true>(w + q * N1);
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int a = 0; a < N1; ++a) {
      const int k2 = t + N1 * q;  // w[q N1 + a] now holds Z[n1 = a][k2]
      const float2 z = k2 == 0 || a == 0 ? w[q * N1 + a] : twmul<true>(w[q * N1 + a], s_tw[a * k2]);
      E[(c * N + a * N2 + k2) * U + u] = z;  // E was last read before the previous barrier
    }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N2; ++j) v[j] = E[(c * N + n1 * N2 + j) * U + u];
  dft<N2, true>(v);
#pragma unroll
  for (int j = 0; j < N2; ++j) out[base_o + (long)c * n + (long)(n1 + N1 * j) * N * N + u] = v[j];
}

template <int N>
int launch_precond_c64_n(pc_ctx *ctx, int nb, int m, const float2 *R, long sr, float2 *W, long sw, const int *act) {
  using PC = PlaneCfg<N>;
  using ZC = ZCfg<N>;
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(fft_plane_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)PC::smem()));
    PC_CK(cudaFuncSetAttribute(fft_plane_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)PC::smem()));
    PC_CK(cudaFuncSetAttribute(fft_zsym_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ZC::smem()));
    PC_CK(cudaFuncSetAttribute(fft_zsym_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ZC::smem()));
    configured = true;
  }
  const float2 *tw = ctx->twf.as<float2>();
  const int lap = ctx->opts.precond == PC_PRECOND_LAPLACIAN;
  fft_plane_kernel<N, true><<<dim3(3 * N / PC::P, m, nb), PC::THREADS, PC::smem(), ctx->stream>>>(R, sr, W, sw, tw,
                                                                                                  act);
  PC_CK_LAUNCH();
  if (ctx->lat)
    fft_zsym_kernel<N, true><<<dim3(N * N / ZC::U, m, nb), ZC::THREADS, ZC::smem(), ctx->stream>>>(
        W, sw, W, sw, tw, ctx->symd.as<double2>(), ctx->kparam.as<KParam>(), act, lap);
  else
    fft_zsym_kernel<N, false><<<dim3(N * N / ZC::U, m, nb), ZC::THREADS, ZC::smem(), ctx->stream>>>(
        W, sw, W, sw, tw, ctx->symd.as<double2>(), ctx->kparam.as<KParam>(), act, lap);
  PC_CK_LAUNCH();
  fft_plane_kernel<N, false><<<dim3(3 * N / PC::P, m, nb), PC::THREADS, PC::smem(), ctx->stream>>>(W, sw, W, sw, tw,
                                                                                                   act);
  PC_CK_LAUNCH();
  return PC_OK;
}

}  // namespace

// complex64 path for 8 <= N <= 128 (cube and general lattice); PC_EUNSUPPORTED for other sizes
int launch_precond_c64(pc_ctx *ctx, int nb, int m, const void *R, long sr, void *W, long sw, const int *act) {
  const float2 *Rf = static_cast<const float2 *>(R);
  float2 *Wf = static_cast<float2 *>(W);
  switch (ctx->N) {
    case 8: return launch_precond_c64_n<8>(ctx, nb, m, Rf, sr, Wf, sw, act);
    case 16: return launch_precond_c64_n<16>(ctx, nb, m, Rf, sr, Wf, sw, act);
    case 32: return launch_precond_c64_n<32>(ctx, nb, m, Rf, sr, Wf, sw, act);
    case 64: return launch_precond_c64_n<64>(ctx, nb, m, Rf, sr, Wf, sw, act);
    case 128: return launch_precond_c64_n<128>(ctx, nb, m, Rf, sr, Wf, sw, act);
    default: return PC_EUNSUPPORTED;
  }
}

}  // namespace pc
