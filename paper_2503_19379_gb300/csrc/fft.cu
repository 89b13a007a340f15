// FFT-diagonalised preconditioner solve W = P^{-1} R (Section 5.2, Algorithm 5.1) with the 3x3 mode symbol of
// eq. penalised_marix, for batches of k-points x fields.
//
// Every circulant K_i, L_i is diagonal in the DFT basis (eq. diag_of_circ), so per mode m the preconditioner
// P = A A' + gamma B'B is the 3x3 matrix sigma I + (gamma - 1) conj(d) d^T with d_i = symbol of D_i on mode m_i and
// sigma = |d|^2. On a general lattice d_i is the symbol of D_hat_i = sum_j b_ji K_j + i L_i, which depends on all
// three mode indices (the same 3x3 algebra holds for any complex d). Its exact inverse (Sherman-Morrison) is (1/sigma) [I - (gamma-1)/(gamma sigma) conj(d) d^T]; with
// the vector-Laplacian variant (gamma -> 1 in P) it is the scalar 1/sigma of Algorithm 5.1.
//
// Passes (each a read and a write of the block):
//   1. forward FFT along x (decimation in frequency: natural order in, bit-reversed mode order out)
//   2. forward FFT along y (same); 1 and 2 run as one plane kernel when an N x N plane fits in shared memory
//   3. along z, for all three components of a column at once: forward DIF FFT, the 3x3 symbol inverse at the mode
//      (bitrev x, bitrev y, bitrev z) times 1/N^3, inverse FFT (decimation in time: bit-reversed in, natural out)
//   4. inverse FFT along y (DIT), 5. inverse FFT along x (DIT); again one plane kernel when the plane fits.
// The frequency data never needs reordering: the DIT inverse consumes the DIF output order directly.
// Each line is transformed in shared memory with radix-2 butterflies; twiddles exp(-2 pi i t / N) come from a
// table computed once on the host.
#include <cmath>

#include "pc_internal.cuh"

namespace pc {

__device__ __forceinline__ int bitrev(int p, int logN) { return (int)(__brev((unsigned)p) >> (32 - logN)); }

// In-place radix-2 FFTs of `lines` lines of length N held in shared memory. Line l = g * lpg + u (group g, member
// u) starts at g * gs + u * ls and its element t sits t * es further. Forward = DIF with exp(-), inverse = DIT with
// exp(+).
// LINE_MAJOR: consecutive threads take consecutive lines (for lines that are adjacent in memory, ls = 1, so that a
// warp reads consecutive addresses); otherwise consecutive butterflies of one line (for contiguous lines, es = 1).
template <typename C, bool FWD, bool LINE_MAJOR = false>
__device__ __forceinline__ void fft_lines(C *a, int lines, int lpg, int gs, int ls, int es, int logN, const C *tw) {
  const int N = 1 << logN, halfN = N >> 1;
  const int total = lines * halfN;
  if (FWD) {
    for (int lh = logN - 1; lh >= 0; --lh) {
      const int half = 1 << lh;
      for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int l = LINE_MAJOR ? q % lines : q / halfN, r = LINE_MAJOR ? q / lines : q - l * halfN;
        const int g = r >> lh, jj = r & (half - 1);
        const int lg = l / lpg, lu = l - lg * lpg;
        const int i0 = lg * gs + lu * ls + ((g << (lh + 1)) + jj) * es, i1 = i0 + half * es;
        const C x0 = a[i0], x1 = a[i1];
        a[i0] = cadd(x0, x1);
        a[i1] = cmul(csub(x0, x1), tw[jj << (logN - 1 - lh)]);
      }
      __syncthreads();
    }
  } else {
    for (int lh = 0; lh < logN; ++lh) {
      const int half = 1 << lh;
      for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int l = LINE_MAJOR ? q % lines : q / halfN, r = LINE_MAJOR ? q / lines : q - l * halfN;
        const int g = r >> lh, jj = r & (half - 1);
        const int lg = l / lpg, lu = l - lg * lpg;
        const int i0 = lg * gs + lu * ls + ((g << (lh + 1)) + jj) * es, i1 = i0 + half * es;
        const C w = tw[jj << (logN - 1 - lh)];
        const C t = cmulc(w, a[i1]);  // conj(w) * a[i1]
        const C x0 = a[i0];
        a[i1] = csub(x0, t);
        a[i0] = cadd(x0, t);
      }
      __syncthreads();
    }
  }
}

template <typename C> __device__ __forceinline__ void load_tw(C *s_tw, const C *tw, int halfN) {
  for (int i = threadIdx.x; i < halfN; i += blockDim.x) s_tw[i] = tw[i];
}

// Pass along x: R rows of N contiguous elements per CTA. grid (3N^2/R, m, nb).
template <typename T, bool FWD>
__global__ void __launch_bounds__(256) fft_x_kernel(const cplx<T> *__restrict__ in, long si, cplx<T> *__restrict__ out,
                                                    long so, const cplx<T> *__restrict__ tw, const int *act, int logN,
                                                    int R) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN;
  C *s_tw = reinterpret_cast<C *>(smem_raw);
  C *a = s_tw + N / 2;
  const long n = 1L << (3 * logN);
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const long base_i = (long)b * si + (long)blockIdx.y * 3 * n + (long)blockIdx.x * R * N;
  const long base_o = (long)b * so + (long)blockIdx.y * 3 * n + (long)blockIdx.x * R * N;
  load_tw(s_tw, tw, N / 2);
  for (int i = threadIdx.x; i < R * N; i += blockDim.x) a[i] = in[base_i + i];
  __syncthreads();
  fft_lines<C, FWD>(a, R, R, 0, N, 1, logN, s_tw);
  for (int i = threadIdx.x; i < R * N; i += blockDim.x) out[base_o + i] = a[i];
}

// Pass along y: a tile of U contiguous x values by N y values, for one (component, z). grid (3*N*(N/U), m, nb).
template <typename T, bool FWD>
__global__ void __launch_bounds__(256) fft_y_kernel(const cplx<T> *__restrict__ in, long si, cplx<T> *__restrict__ out,
                                                    long so, const cplx<T> *__restrict__ tw, const int *act, int logN,
                                                    int U) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN;
  C *s_tw = reinterpret_cast<C *>(smem_raw);
  C *a = s_tw + N / 2;  // [y][u]
  const long n = 1L << (3 * logN);
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int tilesX = N / U;
  const int xt = blockIdx.x % tilesX, plane = blockIdx.x / tilesX;  // plane = comp * N + z
  const long off = (long)blockIdx.y * 3 * n + (long)plane * N * N + (long)xt * U;
  const long base_i = (long)b * si + off, base_o = (long)b * so + off;
  load_tw(s_tw, tw, N / 2);
  for (int i = threadIdx.x; i < N * U; i += blockDim.x) {
    const int y = i / U, u = i - y * U;
    a[i] = in[base_i + (long)y * N + u];
  }
  __syncthreads();
  fft_lines<C, FWD, true>(a, U, U, 0, 1, U, logN, s_tw);
  for (int i = threadIdx.x; i < N * U; i += blockDim.x) {
    const int y = i / U, u = i - y * U;
    out[base_o + (long)y * N + u] = a[i];
  }
}

// Both in-plane transforms of one (component, z) plane held in shared memory: forward = x then y (DIF), inverse =
// y then x (DIT). grid (3N, m, nb). Replaces the separate x and y passes when N^2 elements fit.
template <typename T, bool FWD>
__global__ void __launch_bounds__(512) fft_xy_kernel(const cplx<T> *__restrict__ in, long si, cplx<T> *__restrict__ out,
                                                     long so, const cplx<T> *__restrict__ tw, const int *act,
                                                     int logN) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN;
  C *s_tw = reinterpret_cast<C *>(smem_raw);
  C *a = s_tw + N / 2;  // [y][x]
  const long n = 1L << (3 * logN);
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const long off = (long)blockIdx.y * 3 * n + (long)blockIdx.x * N * N;  // plane = comp * N + z
  const C *src = in + (long)b * si + off;
  C *dst = out + (long)b * so + off;
  load_tw(s_tw, tw, N / 2);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) a[i] = src[i];
  __syncthreads();
  if (FWD) {
    fft_lines<C, true>(a, N, N, 0, N, 1, logN, s_tw);        // rows (x)
    fft_lines<C, true, true>(a, N, N, 0, 1, N, logN, s_tw);  // columns (y), line-major
  } else {
    fft_lines<C, false, true>(a, N, N, 0, 1, N, logN, s_tw);
    fft_lines<C, false>(a, N, N, 0, N, 1, logN, s_tw);
  }
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) dst[i] = a[i];
}

// Pass along z with the symbol: all 3 components of U contiguous x values at one y. grid (N*(N/U), m, nb).
// LAT (general lattice, Section 4.2.2): d_i = sum_j (part of axis j)(m_j) from the tables [b][i][j][N].
template <typename T, bool LAT>
__global__ void __launch_bounds__(256) fft_z_symbol_kernel(const cplx<T> *__restrict__ in, long si,
                                                           cplx<T> *__restrict__ out, long so,
                                                           const cplx<T> *__restrict__ tw,
                                                           const double2 *__restrict__ sym,
                                                           const KParam *__restrict__ kp, const int *act, int logN,
                                                           int U, int laplacian) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN;
  C *s_tw = reinterpret_cast<C *>(smem_raw);
  C *a = s_tw + N / 2;  // [comp][z][u]
  const long n = 1L << (3 * logN);
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int tilesX = N / U;
  const int xt = blockIdx.x % tilesX, y = blockIdx.x / tilesX;
  const long off = (long)blockIdx.y * 3 * n + (long)y * N + (long)xt * U;
  const long base_i = (long)b * si + off, base_o = (long)b * so + off;
  load_tw(s_tw, tw, N / 2);
  for (int i = threadIdx.x; i < 3 * N * U; i += blockDim.x) {
    const int u = i % U, z = (i / U) % N, comp = i / (U * N);
    a[i] = in[base_i + comp * n + (long)z * N * N + u];
  }
  __syncthreads();
  fft_lines<C, true, true>(a, 3 * U, U, N * U, 1, U, logN, s_tw);  // lines (comp, u); z stride U
  // symbol inverse per mode
  const double2 *symb = sym + (long)b * (LAT ? 9 : 3) * N;
  const T fac = (T)((kp[b].gamma - 1.0) / kp[b].gamma);  // (gamma - 1) / gamma, once per block
  const T scale = (T)(1.0 / (double)n);
  const int my = bitrev(y, logN);
  const double2 d2d = LAT ? make_double2(0.0, 0.0) : symb[N + my];
  for (int i = threadIdx.x; i < N * U; i += blockDim.x) {
    const int u = i % U, z = i / U;
    const int mx = bitrev(xt * U + u, logN), mz = bitrev(z, logN);
    C d1, d2, d3;
    if constexpr (LAT) {
      auto dsum = [&](int c) {
        const double2 *t = symb + (long)c * 3 * N;
        const double2 px = t[mx], py = t[N + my], pz = t[2 * N + mz];
        return cmake<C>((T)(px.x + py.x + pz.x), (T)(px.y + py.y + pz.y));
      };
      d1 = dsum(0);
      d2 = dsum(1);
      d3 = dsum(2);
    } else {
      const double2 d1d = symb[mx], d3d = symb[2 * N + mz];
      d1 = cmake<C>((T)d1d.x, (T)d1d.y);
      d2 = cmake<C>((T)d2d.x, (T)d2d.y);
      d3 = cmake<C>((T)d3d.x, (T)d3d.y);
    }
    const T sigma = d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y + d3.x * d3.x + d3.y * d3.y;
    C r1 = a[i], r2 = a[N * U + i], r3 = a[2 * N * U + i];
    if (!(sigma > (T)0)) {
      r1 = r2 = r3 = cmake<C>((T)0, (T)0);
    } else {
      const T inv = scale / sigma;
      if (!laplacian) {
        const C s = cadd(cadd(cmul(d1, r1), cmul(d2, r2)), cmul(d3, r3));  // d^T r
        const T f = fac / sigma;
        r1 = csub(r1, cscale(cmulc(d1, s), f));  // conj(d1) * s
        r2 = csub(r2, cscale(cmulc(d2, s), f));
        r3 = csub(r3, cscale(cmulc(d3, s), f));
      }
      r1 = cscale(r1, inv);
      r2 = cscale(r2, inv);
      r3 = cscale(r3, inv);
    }
    a[i] = r1;
    a[N * U + i] = r2;
    a[2 * N * U + i] = r3;
  }
  __syncthreads();
  fft_lines<C, false, true>(a, 3 * U, U, N * U, 1, U, logN, s_tw);
  for (int i = threadIdx.x; i < 3 * N * U; i += blockDim.x) {
    const int u = i % U, z = (i / U) % N, comp = i / (U * N);
    out[base_o + comp * n + (long)z * N * N + u] = a[i];
  }
}

// ------------------------------------------------------------------------------------------------ register path
// complex64, N = 2^LOGN <= 64: one thread per line with the whole line in registers; shared memory only carries the
// transposes between the passes. Same butterflies and orders as fft_lines (DIF: natural in, bit-reversed out;
// DIT inverse: bit-reversed in, natural out), with the loop structure resolved at compile time.
template <int LOGN, int LH>
__device__ __forceinline__ void reg_dif_stage(float2 (&v)[1 << LOGN], const float2 (&w)[(1 << LOGN) / 2]) {
  constexpr int half = 1 << LH;
#pragma unroll
  for (int r = 0; r < (1 << LOGN) / 2; ++r) {
    const int j = r & (half - 1), i0 = ((r >> LH) << (LH + 1)) + j, i1 = i0 + half;
    const float2 x0 = v[i0], x1 = v[i1];
    v[i0] = cadd(x0, x1);
    v[i1] = j == 0 ? csub(x0, x1) : cmul(csub(x0, x1), w[j << (LOGN - 1 - LH)]);  // w[0] = 1
  }
  if constexpr (LH > 0) reg_dif_stage<LOGN, LH - 1>(v, w);
}
template <int LOGN, int LH>
__device__ __forceinline__ void reg_dit_stage(float2 (&v)[1 << LOGN], const float2 (&w)[(1 << LOGN) / 2]) {
  constexpr int half = 1 << LH;
#pragma unroll
  for (int r = 0; r < (1 << LOGN) / 2; ++r) {
    const int j = r & (half - 1), i0 = ((r >> LH) << (LH + 1)) + j, i1 = i0 + half;
    const float2 t = j == 0 ? v[i1] : cmulc(w[j << (LOGN - 1 - LH)], v[i1]);
    const float2 x0 = v[i0];
    v[i1] = csub(x0, t);
    v[i0] = cadd(x0, t);
  }
  if constexpr (LH + 1 < LOGN) reg_dit_stage<LOGN, LH + 1>(v, w);
}
template <int LOGN>
__device__ __forceinline__ void reg_dif(float2 (&v)[1 << LOGN], const float2 (&w)[(1 << LOGN) / 2]) {
  reg_dif_stage<LOGN, LOGN - 1>(v, w);
}
template <int LOGN>
__device__ __forceinline__ void reg_dit_inv(float2 (&v)[1 << LOGN], const float2 (&w)[(1 << LOGN) / 2]) {
  reg_dit_stage<LOGN, 0>(v, w);
}
template <int LOGN> __device__ __forceinline__ void reg_twiddles(float2 (&w)[(1 << LOGN) / 2], const float2 *tw) {
#pragma unroll
  for (int i = 0; i < (1 << LOGN) / 2; ++i) w[i] = tw[i];
}

// Both in-plane transforms of P = min(256 / N, N) planes (component, z): rows (x) then columns (y) forward, columns
// then rows inverse. Plane rows are padded to N + 1 elements so that row-wise and column-wise line reads are free of
// bank conflicts. grid (3N / P, m, nb), P N threads; thread t owns line t % N of plane t / N.
template <int LOGN> constexpr int xy_planes() { return (256 >> LOGN) < (1 << LOGN) ? (256 >> LOGN) : (1 << LOGN); }
template <int LOGN, bool FWD>
__global__ void __launch_bounds__(xy_planes<LOGN>() * (1 << LOGN)) fft_xy_reg_kernel(const float2 *__restrict__ in, long si,
                                                         float2 *__restrict__ out, long so,
                                                         const float2 *__restrict__ tw, const int *act) {
  constexpr int N = 1 << LOGN, P = xy_planes<LOGN>(), LD = N + 1, NT = P * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *a = reinterpret_cast<float2 *>(smem_raw);  // [P][N][LD]
  const long n = (long)N * N * N;
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const long off = (long)blockIdx.y * 3 * n + (long)blockIdx.x * P * N * N;
  const float2 *src = in + (long)b * si + off;
  float2 *dst = out + (long)b * so + off;
  float2 w[N / 2];
  reg_twiddles<LOGN>(w, tw);
  for (int i = threadIdx.x; i < P * N * N; i += NT) {
    const int x = i % N, py = i / N;  // py = plane * N + y
    a[py * LD + x] = src[i];
  }
  __syncthreads();
  const int pl = threadIdx.x / N, l = threadIdx.x % N;
  float2 *ap = a + pl * N * LD;
  float2 v[N];
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const bool rows = FWD ? pass == 0 : pass == 1;  // row lines: x varies, fixed y = l
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = rows ? ap[l * LD + i] : ap[i * LD + l];
    if (FWD)
      reg_dif<LOGN>(v, w);
    else
      reg_dit_inv<LOGN>(v, w);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (rows)
        ap[l * LD + i] = v[i];
      else
        ap[i * LD + l] = v[i];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < P * N * N; i += NT) {
    const int x = i % N, py = i / N;
    dst[i] = a[py * LD + x];
  }
}

// Along z with the symbol: YP rows y (YP * 3 * N threads, one per (y, component, x) line), all x. The forward DIF
// along z, the 3x3 symbol inverse per mode (components exchanged through shared memory) and the inverse DIT.
// grid (N / YP, m, nb).
template <int LOGN, int YP>
__global__ void __launch_bounds__(YP * 3 * (1 << LOGN)) fft_z_reg_kernel(const float2 *__restrict__ in, long si,
                                                                        float2 *__restrict__ out, long so,
                                                                        const float2 *__restrict__ tw,
                                                                        const double2 *__restrict__ sym,
                                                                        const KParam *__restrict__ kp,
                                                                        const int *act, int laplacian) {
  constexpr int N = 1 << LOGN, NT = YP * 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *a = reinterpret_cast<float2 *>(smem_raw);  // [YP][3][N z][N x]
  float2 *s1 = a + YP * 3 * N * N;                   // symbols d1 (x), d2 (y), d3 (z) in FP32: [3][N]
  const long n = (long)N * N * N;
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int y0 = blockIdx.x * YP;
  const long base_i = (long)b * si + (long)blockIdx.y * 3 * n + (long)y0 * N;
  const long base_o = (long)b * so + (long)blockIdx.y * 3 * n + (long)y0 * N;
  const double2 *symb = sym + (long)b * 3 * N;
  for (int i = threadIdx.x; i < 3 * N; i += NT) s1[i] = make_float2((float)symb[i].x, (float)symb[i].y);
  float2 w[N / 2];
  reg_twiddles<LOGN>(w, tw);
  // a[yy][c][z][x] <- in[c n + z N^2 + (y0 + yy) N + x]
  for (int i = threadIdx.x; i < YP * 3 * N * N; i += NT) {
    const int x = i % N, z = (i / N) % N, c = (i / (N * N)) % 3, yy = i / (3 * N * N);
    a[i] = in[base_i + (long)c * n + (long)z * N * N + (long)yy * N + x];
  }
  __syncthreads();
  const int x = threadIdx.x % N, line = threadIdx.x / N;  // line = yy * 3 + c
  float2 *al = a + (long)line * N * N + x;
  float2 v[N];
#pragma unroll
  for (int z = 0; z < N; ++z) v[z] = al[z * N];
  reg_dif<LOGN>(v, w);
#pragma unroll
  for (int z = 0; z < N; ++z) al[z * N] = v[z];
  __syncthreads();
  const float fac = kp[b].pfacf;  // (gamma - 1) / gamma
  const float scale = 1.0f / (float)n;
  for (int i = threadIdx.x; i < YP * N * N; i += NT) {
    const int xx = i % N, z = (i / N) % N, yy = i / (N * N);
    const float2 d1 = s1[bitrev(xx, LOGN)], d2 = s1[N + bitrev(y0 + yy, LOGN)], d3 = s1[2 * N + bitrev(z, LOGN)];
    const float sigma = d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y + d3.x * d3.x + d3.y * d3.y;
    float2 *e = a + (long)yy * 3 * N * N + z * N + xx;
    float2 r1 = e[0], r2 = e[N * N], r3 = e[2 * N * N];
    if (!(sigma > 0.f)) {
      r1 = r2 = r3 = make_float2(0.f, 0.f);
    } else {
      const float inv = scale / sigma;
      if (!laplacian) {
        const float2 sd = cadd(cadd(cmul(d1, r1), cmul(d2, r2)), cmul(d3, r3));  // d^T r
        const float f = fac / sigma;
        r1 = csub(r1, cscale(cmulc(d1, sd), f));
        r2 = csub(r2, cscale(cmulc(d2, sd), f));
        r3 = csub(r3, cscale(cmulc(d3, sd), f));
      }
      r1 = cscale(r1, inv);
      r2 = cscale(r2, inv);
      r3 = cscale(r3, inv);
    }
    e[0] = r1;
    e[N * N] = r2;
    e[2 * N * N] = r3;
  }
  __syncthreads();
#pragma unroll
  for (int z = 0; z < N; ++z) v[z] = al[z * N];
  reg_dit_inv<LOGN>(v, w);
#pragma unroll
  for (int z = 0; z < N; ++z) al[z * N] = v[z];
  __syncthreads();
  for (int i = threadIdx.x; i < YP * 3 * N * N; i += NT) {
    const int xx = i % N, z = (i / N) % N, c = (i / (N * N)) % 3, yy = i / (3 * N * N);
    out[base_o + (long)c * n + (long)z * N * N + (long)yy * N + xx] = a[i];
  }
}

template <int LOGN>
static int launch_precond_reg(pc_ctx *ctx, int nb, int m, const float2 *R, long sr, float2 *W, long sw,
                              const int *act) {
  constexpr int N = 1 << LOGN, P = xy_planes<LOGN>();
  constexpr int YP = N >= 64 ? 1 : (N >= 32 ? 2 : (N >= 16 ? 4 : 8));
  const size_t sxy = sizeof(float2) * (size_t)P * N * (N + 1);
  const size_t sz = sizeof(float2) * ((size_t)YP * 3 * N * N + 3 * N);
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(fft_xy_reg_kernel<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sxy));
    PC_CK(cudaFuncSetAttribute(fft_xy_reg_kernel<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sxy));
    PC_CK(cudaFuncSetAttribute(fft_z_reg_kernel<LOGN, YP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz));
    configured = true;
  }
  const float2 *tw = ctx->twf.as<float2>();
  const int lap = ctx->opts.precond == PC_PRECOND_LAPLACIAN;
  fft_xy_reg_kernel<LOGN, true><<<dim3(3 * N / P, m, nb), P * N, sxy, ctx->stream>>>(R, sr, W, sw, tw, act);
  PC_CK_LAUNCH();
  fft_z_reg_kernel<LOGN, YP><<<dim3(N / YP, m, nb), YP * 3 * N, sz, ctx->stream>>>(
      W, sw, W, sw, tw, ctx->symd.as<double2>(), ctx->kparam.as<KParam>(), act, lap);
  PC_CK_LAUNCH();
  fft_xy_reg_kernel<LOGN, false><<<dim3(3 * N / P, m, nb), P * N, sxy, ctx->stream>>>(W, sw, W, sw, tw, act);
  PC_CK_LAUNCH();
  return PC_OK;
}

template <typename T>
static int launch_precond_t(pc_ctx *ctx, int nb, int m, const void *R, long sr, void *W, long sw, const int *act) {
  using C = cplx<T>;
  const int N = ctx->N, logN = ctx->logN;
  const C *tw = std::is_same<T, double>::value ? ctx->twd.as<C>() : ctx->twf.as<C>();
  const int elems = 2048;
  const int Rr = std::min(elems / N, N * N);          // rows per CTA along x
  const int Uy = std::min(N, std::max(1, elems / N));  // x values per CTA along y
  int Uz = 1;
  while (Uz * 2 <= N && 3 * N * Uz * 2 <= 3 * elems / 2) Uz *= 2;
  const size_t tw_b = sizeof(C) * (N / 2);
  const size_t sx = tw_b + sizeof(C) * Rr * N, sy = tw_b + sizeof(C) * Uy * N, sz = tw_b + sizeof(C) * 3 * N * Uz;
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(fft_x_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    PC_CK(cudaFuncSetAttribute(fft_x_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    PC_CK(cudaFuncSetAttribute(fft_y_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    PC_CK(cudaFuncSetAttribute(fft_y_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    PC_CK(cudaFuncSetAttribute(fft_z_symbol_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    PC_CK(cudaFuncSetAttribute(fft_z_symbol_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
  const C *Rc = static_cast<const C *>(R);
  C *Wc = static_cast<C *>(W);
  const unsigned gx = (unsigned)(3 * N * N / Rr), gy = (unsigned)(3 * N * (N / Uy)), gz = (unsigned)(N * (N / Uz));
  const size_t sxy = tw_b + sizeof(C) * (size_t)N * N;
  const bool plane = sxy <= 200 * 1024;  // both in-plane transforms in one pass
  static bool configured_xy = false;
  if (plane && !configured_xy) {
    PC_CK(cudaFuncSetAttribute(fft_xy_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    PC_CK(cudaFuncSetAttribute(fft_xy_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured_xy = true;
  }
  const int txy = N * N >= 4096 ? 512 : 256;
  if (plane) {
    fft_xy_kernel<T, true><<<dim3(3 * N, m, nb), txy, sxy, ctx->stream>>>(Rc, sr, Wc, sw, tw, act, logN);
    PC_CK_LAUNCH();
  } else {
    fft_x_kernel<T, true><<<dim3(gx, m, nb), 256, sx, ctx->stream>>>(Rc, sr, Wc, sw, tw, act, logN, Rr);
    PC_CK_LAUNCH();
    fft_y_kernel<T, true><<<dim3(gy, m, nb), 256, sy, ctx->stream>>>(Wc, sw, Wc, sw, tw, act, logN, Uy);
    PC_CK_LAUNCH();
  }
  const int lap = ctx->opts.precond == PC_PRECOND_LAPLACIAN;
  if (ctx->lat)
    fft_z_symbol_kernel<T, true><<<dim3(gz, m, nb), 256, sz, ctx->stream>>>(
        Wc, sw, Wc, sw, tw, ctx->symd.as<double2>(), ctx->kparam.as<KParam>(), act, logN, Uz, lap);
  else
    fft_z_symbol_kernel<T, false><<<dim3(gz, m, nb), 256, sz, ctx->stream>>>(
        Wc, sw, Wc, sw, tw, ctx->symd.as<double2>(), ctx->kparam.as<KParam>(), act, logN, Uz, lap);
  PC_CK_LAUNCH();
  if (plane) {
    fft_xy_kernel<T, false><<<dim3(3 * N, m, nb), txy, sxy, ctx->stream>>>(Wc, sw, Wc, sw, tw, act, logN);
    PC_CK_LAUNCH();
  } else {
    fft_y_kernel<T, false><<<dim3(gy, m, nb), 256, sy, ctx->stream>>>(Wc, sw, Wc, sw, tw, act, logN, Uy);
    PC_CK_LAUNCH();
    fft_x_kernel<T, false><<<dim3(gx, m, nb), 256, sx, ctx->stream>>>(Wc, sw, Wc, sw, tw, act, logN, Rr);
    PC_CK_LAUNCH();
  }
  return PC_OK;
}

int launch_precond(pc_ctx *ctx, int nb, int m, int dtype, const void *R, long sr, void *W, long sw,
                   const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  if (dtype == PC_C128) return launch_precond_t<double>(ctx, nb, m, R, sr, W, sw, act);
  {
    const int rc = launch_precond_c64(ctx, nb, m, R, sr, W, sw, act);  // fft_c64.cu: N <= 128, cube and lattice
    if (rc != PC_EUNSUPPORTED) return rc;
  }
  // the register path's symbols are per axis; a general lattice takes the shared-memory path
  if (ctx->lat) return launch_precond_t<float>(ctx, nb, m, R, sr, W, sw, act);
  const float2 *Rf = static_cast<const float2 *>(R);
  float2 *Wf = static_cast<float2 *>(W);
  switch (ctx->logN) {
    case 3: return launch_precond_reg<3>(ctx, nb, m, Rf, sr, Wf, sw, act);
    case 4: return launch_precond_reg<4>(ctx, nb, m, Rf, sr, Wf, sw, act);
    case 5: return launch_precond_reg<5>(ctx, nb, m, Rf, sr, Wf, sw, act);
    case 6: return launch_precond_reg<6>(ctx, nb, m, Rf, sr, Wf, sw, act);
    default: return launch_precond_t<float>(ctx, nb, m, R, sr, W, sw, act);
  }
}

}  // namespace pc

using namespace pc;

extern "C" int pc_apply_precond(pc_ctx *ctx, int nb, const double *kpts, const double *gammas, int m, int dtype,
                                const void *R, void *W) {
  PC_REQUIRE(ctx && kpts && gammas && R && W, "pc_apply_precond: null argument");
  PC_REQUIRE(nb >= 0 && m >= 0, "pc_apply_precond: negative size");
  PC_REQUIRE(dtype == PC_C128 || dtype == PC_C64, "pc_apply_precond: bad dtype %d", dtype);
  int rc = upload_kpoints(ctx, nb, kpts, gammas);
  if (rc) return rc;
  const long blk = (long)m * 3 * ctx->n;
  return launch_precond(ctx, nb, m, dtype, R, blk, W, blk, nullptr);
}
