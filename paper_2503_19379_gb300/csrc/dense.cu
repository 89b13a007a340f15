// Tall-skinny block kernels of LOBPCG (Section 5.1): Gram products A^H B, block updates S C, residuals
// R = AX - X Theta with column norms, the k = 0 projection of the constant fields, and the counter-based initial
// blocks. Blocks are column-major: column j of a block with L rows starts at j * L.
#include <cmath>
#include <mutex>

#include "dfloat.cuh"
#include "pc_internal.cuh"

namespace pc {

// ------------------------------------------------------------------------------------------------ Gram
// Partial products over a chunk of rows; grid (nchunk, 1, nb). Thread (ty, tx) of a 16 x 16 block accumulates the
// outputs (ty + 16 r, tx + 16 s), r, s < 4, so p, q <= 64.
constexpr int GRAM_TL = 16;

template <typename T>
__global__ void __launch_bounds__(256) gram_partial_kernel(const cplx<T> *__restrict__ A, long sa,
                                                          const cplx<T> *__restrict__ B, long sb, long L, int p,
                                                          int q, long chunk, double2 *__restrict__ part,
                                                          const int *__restrict__ act) {
  // operands and per-chunk sums in the input precision T; chunks are summed in FP64 by gram_reduce_kernel
  using C = cplx<T>;
  __shared__ C As[64][GRAM_TL + 1];
  __shared__ C Bs[64][GRAM_TL + 1];
  const int bi = blockIdx.z;
  const int b = act ? act[bi] : bi;
  const C *Ab = A + (long)b * sa;
  const C *Bb = B + (long)b * sb;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  C acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[r][s] = cmake<C>((T)0, (T)0);
  const long beg = (long)blockIdx.x * chunk, end = min(L, beg + chunk);
  for (long l0 = beg; l0 < end; l0 += GRAM_TL) {
    for (int i = threadIdx.x; i < 64 * GRAM_TL; i += 256) {
      const int col = i / GRAM_TL, t = i - col * GRAM_TL;
      const long l = l0 + t;
      C va = cmake<C>((T)0, (T)0), vb = va;
      if (l < end) {
        if (col < p) va = Ab[(long)col * L + l];
        if (col < q) vb = Bb[(long)col * L + l];
      }
      As[col][t] = va;
      Bs[col][t] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < GRAM_TL; ++t) {
      C a[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[ty + 16 * r][t];
#pragma unroll
      for (int s = 0; s < 4; ++s) bv[s] = Bs[tx + 16 * s][t];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          acc[r][s].x = fma(a[r].x, bv[s].x, fma(a[r].y, bv[s].y, acc[r][s].x));
          acc[r][s].y = fma(a[r].x, bv[s].y, fma(-a[r].y, bv[s].x, acc[r][s].y));
        }
    }
    __syncthreads();
  }
  double2 *o = part + ((long)bi * gridDim.x + blockIdx.x) * p * q;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = ty + 16 * r, j = tx + 16 * s;
      if (i < p && j < q) o[i * q + j] = cmake<double2>((double)acc[r][s].x, (double)acc[r][s].y);
    }
}

// General p x q product with the thread tile sized to the output: block (ceil(q/R), ceil(p/R)), R x R per thread.
template <typename T, int R>
__global__ void __launch_bounds__(256) gram_tile_partial_kernel(const cplx<T> *__restrict__ A, long sa,
                                                               const cplx<T> *__restrict__ B, long sb, long L, int p,
                                                               int q, long chunk, double2 *__restrict__ part,
                                                               const int *__restrict__ act) {
  using C = cplx<T>;
  __shared__ C As[64][GRAM_TL + 1];
  __shared__ C Bs[64][GRAM_TL + 1];
  const int bi = blockIdx.z;
  const int b = act ? act[bi] : bi;
  const C *Ab = A + (long)b * sa;
  const C *Bb = B + (long)b * sb;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * blockDim.x + tx, nthr = blockDim.x * blockDim.y;
  C acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = cmake<C>((T)0, (T)0);
  const long beg = (long)blockIdx.x * chunk, end = min(L, beg + chunk);
  const int pq = max(p, q);
  for (long l0 = beg; l0 < end; l0 += GRAM_TL) {
    for (int i = tid; i < pq * GRAM_TL; i += nthr) {
      const int col = i / GRAM_TL, t = i - col * GRAM_TL;
      const long l = l0 + t;
      C va = cmake<C>((T)0, (T)0), vb = va;
      if (l < end) {
        if (col < p) va = Ab[(long)col * L + l];
        if (col < q) vb = Bb[(long)col * L + l];
      }
      As[col][t] = va;
      Bs[col][t] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < GRAM_TL; ++t) {
      C a[R], bv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = As[min(ty * R + r, pq - 1)][t];
#pragma unroll
      for (int c = 0; c < R; ++c) bv[c] = Bs[min(tx * R + c, pq - 1)][t];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) {
          acc[r][c].x = fma(a[r].x, bv[c].x, fma(a[r].y, bv[c].y, acc[r][c].x));
          acc[r][c].y = fma(a[r].x, bv[c].y, fma(-a[r].y, bv[c].x, acc[r][c].y));
        }
    }
    __syncthreads();
  }
  double2 *o = part + ((long)bi * gridDim.x + blockIdx.x) * p * q;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int i = ty * R + r, j = tx * R + c;
      if (i < p && j < q) o[i * q + j] = cmake<double2>((double)acc[r][c].x, (double)acc[r][c].y);
    }
}

__global__ void gram_reduce_kernel(const double2 *__restrict__ part, int nchunk, int p, int q,
                                   const int *__restrict__ act, double2 *__restrict__ G, long sg) {
  const int bi = blockIdx.x;
  const int b = act ? act[bi] : bi;
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < p * q; i += gridDim.y * blockDim.x) {
    double2 s = cmake<double2>(0.0, 0.0);
    for (int c = 0; c < nchunk; ++c) s = cadd(s, part[((long)bi * nchunk + c) * p * q + i]);
    G[(long)b * sg + i] = s;
  }
}

static int gram_chunks(int nb, long L) {
  long want = std::max<long>(1, (4L * sm_count() + nb - 1) / std::max(nb, 1));
  long maxc = std::max<long>(1, L / 512);
  return (int)std::min<long>(std::min(want, maxc), 256);
}

// partial sums per k-point that either Gram path may write: the CUDA-core kernels' chunks, or the tensor-core
// kernel's (at least tc_min_chunks)
static int gram_scratch_chunks(int nb, long L) { return std::max(gram_chunks(nb, L), tc_min_chunks(L)); }

size_t gram_scratch_bytes(int nb, long L, int p, int q) {
  return sizeof(double2) * (size_t)nb * gram_scratch_chunks(nb, L) * p * q;
}

int launch_gram(int nb, long L, int p, int q, int dtype, const void *A, long sa, const void *B, long sb, void *G,
                void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc, long sg) {
  if (nb == 0 || p == 0 || q == 0) return PC_OK;
  if (dtype == PC_C64) {
    const int rc = launch_gram_tc(nb, L, p, q, A, sa, B, sb, G, scratch, scratch_bytes, st, act, nb_alloc, sg);
    if (rc != PC_EUNSUPPORTED) return rc;
  }
  const int nchunk = gram_chunks(nb, L);
  if (gram_scratch_bytes(nb, L, p, q) > scratch_bytes) {
    set_error("gram: scratch too small");
    return PC_EINVAL;
  }
  long chunk = (L + nchunk - 1) / nchunk;
  chunk = (chunk + GRAM_TL - 1) / GRAM_TL * GRAM_TL;
  double2 *part = static_cast<double2 *>(scratch);
  const int R = std::max(p, q) <= 32 ? 2 : 4;
  const dim3 blk((q + R - 1) / R, (p + R - 1) / R);
  if (R == 2 && dtype == PC_C128)
    gram_tile_partial_kernel<double, 2><<<dim3(nchunk, 1, nb), blk, 0, st>>>(
        static_cast<const double2 *>(A), sa, static_cast<const double2 *>(B), sb, L, p, q, chunk, part, act);
  else if (R == 2)
    gram_tile_partial_kernel<float, 2><<<dim3(nchunk, 1, nb), blk, 0, st>>>(
        static_cast<const float2 *>(A), sa, static_cast<const float2 *>(B), sb, L, p, q, chunk, part, act);
  else if (dtype == PC_C128)
    gram_partial_kernel<double><<<dim3(nchunk, 1, nb), 256, 0, st>>>(
        static_cast<const double2 *>(A), sa, static_cast<const double2 *>(B), sb, L, p, q, chunk, part, act);
  else
    gram_partial_kernel<float><<<dim3(nchunk, 1, nb), 256, 0, st>>>(
        static_cast<const float2 *>(A), sa, static_cast<const float2 *>(B), sb, L, p, q, chunk, part, act);
  PC_CK_LAUNCH();
  gram_reduce_kernel<<<dim3(nb, (p * q + 255) / 256), 256, 0, st>>>(part, nchunk, p, q, act, static_cast<double2 *>(G),
                                                                    sg > 0 ? sg : (long)p * q);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ------------------------------------------------------------------------------------------------ Gram pair
// G = S^H S and H = S^H (AS) for the same panel S (p <= 64 columns) in one pass over the rows. Both are Hermitian
// (Op is), so only tiles on or above the diagonal are accumulated and the reduction mirrors the rest. Thread
// (ty, tx) of a TD x TD block (TD = ceil(p / R)) owns the R x R output tile at (ty R, tx R); tiles with ty > tx
// only help load.
template <typename T, int R>
__global__ void __launch_bounds__(256) gram_pair_partial_kernel(const cplx<T> *__restrict__ S,
                                                               const cplx<T> *__restrict__ AS, long ss, long L, int p,
                                                               long chunk, double2 *__restrict__ partG,
                                                               double2 *__restrict__ partH,
                                                               const int *__restrict__ act) {
  using C = cplx<T>;
  __shared__ C Ss[64][GRAM_TL + 1];
  __shared__ C As[64][GRAM_TL + 1];
  const int bi = blockIdx.z;
  const int b = act ? act[bi] : bi;
  const C *Sb = S + (long)b * ss;
  const C *Ab = AS + (long)b * ss;
  const int TD = blockDim.x;  // blockDim = (TD, TD)
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TD + tx, nthr = TD * TD;
  const bool active = ty <= tx;
  C g[R][R], hh[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) g[r][c] = hh[r][c] = cmake<C>((T)0, (T)0);
  const long beg = (long)blockIdx.x * chunk, end = min(L, beg + chunk);
  for (long l0 = beg; l0 < end; l0 += GRAM_TL) {
    for (int i = tid; i < p * GRAM_TL; i += nthr) {
      const int col = i / GRAM_TL, t = i - col * GRAM_TL;
      const long l = l0 + t;
      C vs = cmake<C>((T)0, (T)0), va = vs;
      if (l < end) {
        vs = Sb[(long)col * L + l];
        va = Ab[(long)col * L + l];
      }
      Ss[col][t] = vs;
      As[col][t] = va;
    }
    __syncthreads();
    if (active) {
#pragma unroll 2
      for (int t = 0; t < GRAM_TL; ++t) {
        C a[R], bs[R], ba[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = Ss[min(ty * R + r, p - 1)][t];
#pragma unroll
        for (int c = 0; c < R; ++c) {
          const int j = min(tx * R + c, p - 1);
          bs[c] = Ss[j][t];
          ba[c] = As[j][t];
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < R; ++c) {
            g[r][c].x = fma(a[r].x, bs[c].x, fma(a[r].y, bs[c].y, g[r][c].x));
            g[r][c].y = fma(a[r].x, bs[c].y, fma(-a[r].y, bs[c].x, g[r][c].y));
            hh[r][c].x = fma(a[r].x, ba[c].x, fma(a[r].y, ba[c].y, hh[r][c].x));
            hh[r][c].y = fma(a[r].x, ba[c].y, fma(-a[r].y, ba[c].x, hh[r][c].y));
          }
      }
    }
    __syncthreads();
  }
  if (!active) return;
  const long o = ((long)bi * gridDim.x + blockIdx.x) * p * p;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int i = ty * R + r, j = tx * R + c;
      if (i < p && j < p && i <= j) {
        partG[o + i * p + j] = cmake<double2>((double)g[r][c].x, (double)g[r][c].y);
        partH[o + i * p + j] = cmake<double2>((double)hh[r][c].x, (double)hh[r][c].y);
      }
    }
}

// sums the chunks of the upper triangle and mirrors it: G[j][i] = conj(G[i][j])
__global__ void gram_pair_reduce_kernel(const double2 *__restrict__ partG, const double2 *__restrict__ partH,
                                        int nchunk, int p, const int *__restrict__ act, double2 *__restrict__ G,
                                        double2 *__restrict__ H, long sgb) {
  const int bi = blockIdx.x;
  const int b = act ? act[bi] : bi;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < p * p; e += gridDim.y * blockDim.x) {
    const int i = e / p, j = e - i * p;
    if (i > j) continue;
    double2 sg = cmake<double2>(0.0, 0.0), sh = sg;
    for (int c = 0; c < nchunk; ++c) {
      sg = cadd(sg, partG[((long)bi * nchunk + c) * p * p + e]);
      sh = cadd(sh, partH[((long)bi * nchunk + c) * p * p + e]);
    }
    if (i == j) {
      sg.y = 0.0;
      sh.y = 0.0;
    }
    G[(long)b * sgb + i * p + j] = sg;
    H[(long)b * sgb + i * p + j] = sh;
    G[(long)b * sgb + j * p + i] = cmake<double2>(sg.x, -sg.y);
    H[(long)b * sgb + j * p + i] = cmake<double2>(sh.x, -sh.y);
  }
}

size_t gram_pair_scratch_bytes(int nb, long L, int p) {
  return 2 * sizeof(double2) * (size_t)nb * gram_scratch_chunks(nb, L) * p * p;
}

void launch_gram_pair_reduce(int nb, int nchunk, int p, const double2 *part, const int *act, void *G, void *H,
                             cudaStream_t st, long sg) {
  gram_pair_reduce_kernel<<<dim3(nb, (p * p + 255) / 256), 256, 0, st>>>(
      part, part + (size_t)nb * nchunk * p * p, nchunk, p, act, static_cast<double2 *>(G), static_cast<double2 *>(H),
      sg > 0 ? sg : (long)p * p);
}

void launch_gram_reduce(int nb, int nchunk, int p, int q, const double2 *part, const int *act, void *G,
                        cudaStream_t st, long sg) {
  gram_reduce_kernel<<<dim3(nb, (p * q + 255) / 256), 256, 0, st>>>(part, nchunk, p, q, act, static_cast<double2 *>(G),
                                                                    sg > 0 ? sg : (long)p * q);
}

template <typename T>
static int launch_gram_pair_t(int nb, long L, int p, const void *S, const void *AS, long ss, double2 *part,
                              int nchunk, long chunk, cudaStream_t st, const int *act) {
  const cplx<T> *Sc = static_cast<const cplx<T> *>(S);
  const cplx<T> *Ac = static_cast<const cplx<T> *>(AS);
  double2 *pG = part, *pH = part + (size_t)nb * nchunk * p * p;
  if (p <= 32) {
    const int TD = (p + 1) / 2;
    gram_pair_partial_kernel<T, 2><<<dim3(nchunk, 1, nb), dim3(TD, TD), 0, st>>>(Sc, Ac, ss, L, p, chunk, pG, pH, act);
  } else if (p <= 48) {
    const int TD = (p + 2) / 3;
    gram_pair_partial_kernel<T, 3><<<dim3(nchunk, 1, nb), dim3(TD, TD), 0, st>>>(Sc, Ac, ss, L, p, chunk, pG, pH, act);
  } else {
    const int TD = (p + 3) / 4;
    gram_pair_partial_kernel<T, 4><<<dim3(nchunk, 1, nb), dim3(TD, TD), 0, st>>>(Sc, Ac, ss, L, p, chunk, pG, pH, act);
  }
  PC_CK_LAUNCH();
  return PC_OK;
}

int launch_gram_pair(int nb, long L, int p, int dtype, const void *S, const void *AS, long ss, void *G, void *H,
                     void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc, long sg) {
  if (nb == 0 || p == 0) return PC_OK;
  if (p > 64) {
    set_error("gram_pair: at most 64 columns");
    return PC_EINVAL;
  }
  if (gram_pair_scratch_bytes(nb, L, p) > scratch_bytes) {
    set_error("gram_pair: scratch too small");
    return PC_EINVAL;
  }
  if (dtype == PC_C64) {
    const int rc = launch_gram_pair_tc(nb, L, p, S, AS, ss, G, H, scratch, scratch_bytes, st, act, nb_alloc, sg);
    if (rc != PC_EUNSUPPORTED) return rc;
  }
  const int nchunk = gram_chunks(nb, L);
  long chunk = (L + nchunk - 1) / nchunk;
  chunk = (chunk + GRAM_TL - 1) / GRAM_TL * GRAM_TL;
  double2 *part = static_cast<double2 *>(scratch);
  int rc = dtype == PC_C128 ? launch_gram_pair_t<double>(nb, L, p, S, AS, ss, part, nchunk, chunk, st, act)
                            : launch_gram_pair_t<float>(nb, L, p, S, AS, ss, part, nchunk, chunk, st, act);
  if (rc) return rc;
  gram_pair_reduce_kernel<<<dim3(nb, (p * p + 255) / 256), 256, 0, st>>>(
      part, part + (size_t)nb * nchunk * p * p, nchunk, p, act, static_cast<double2 *>(G), static_cast<double2 *>(H),
      sg > 0 ? sg : (long)p * p);
  PC_CK_LAUNCH();
  return PC_OK;
}

size_t gram_pair_coupled_scratch_bytes(int nb, long L, int p, int q2) {
  return std::max({sizeof(double2) * (size_t)nb * gram_scratch_chunks(nb, L) * p * (2 * p + q2),
                   gram_pair_scratch_bytes(nb, L, p), gram_scratch_bytes(nb, L, q2, p)});
}

int launch_gram_pair_coupled(int nb, long L, int p, int q2, int dtype, const void *S, const void *AS, long ss,
                             const void *R, long sr, void *G, void *H, void *RQ, void *scratch, size_t scratch_bytes,
                             cudaStream_t st, const int *act, int nb_alloc, long sg, long srq) {
  if (nb == 0 || p == 0) return PC_OK;
  if (dtype == PC_C64) {
    const int rc = launch_gram_pair_coupled_tc(nb, L, p, q2, S, AS, ss, R, sr, G, H, RQ, scratch, scratch_bytes, st,
                                               act, nb_alloc, sg, srq);
    if (rc != PC_EUNSUPPORTED) return rc;
  }
  int rc = launch_gram_pair(nb, L, p, dtype, S, AS, ss, G, H, scratch, scratch_bytes, st, act, nb_alloc, sg);
  if (rc) return rc;
  return launch_gram(nb, L, q2, p, dtype, R, sr, S, ss, RQ, scratch, scratch_bytes, st, act, nb_alloc, srq);
}

// ------------------------------------------------------------------------------------------------ block update
// Y_b[:, j] = sum_i S_b[:, i] C_b[i, j] (+ Z_b[:, j] when Z is given); grid (ceil(L/256), ceil(q/QB), nb); one row
// per thread, QB outputs. Products and sums run in the precision T of S and Y; Z is a complex64 addend (the
// complex64 correction added to the FP64 block in the mixed-precision update). Each column group re-reads S, so
// the launcher takes the width that covers q in the fewest groups with the fewest idle columns (complex64: one
// group of up to 24 columns, 48 accumulator registers; complex128: 16).
constexpr int UPD_PMAX = 64;

template <typename T, int QB>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
    block_update_kernel(const cplx<T> *__restrict__ S, long ss, const double2 *__restrict__ Cm, long sc,
                        cplx<T> *__restrict__ Y, long sy, const float2 *__restrict__ Z, long sz, long L, int p, int q,
                        const int *__restrict__ act) {
  using C = cplx<T>;
  __shared__ C Cs[UPD_PMAX][QB];
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int j0 = blockIdx.y * QB;
  const double2 *Cb = Cm + (long)b * sc;
  for (int i = threadIdx.x; i < p * QB; i += blockDim.x) {
    const int r = i / QB, c = i - r * QB;
    const double2 v = (j0 + c < q) ? Cb[r * q + j0 + c] : cmake<double2>(0.0, 0.0);
    Cs[r][c] = cmake<C>((T)v.x, (T)v.y);
  }
  __syncthreads();
  const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const C *Sb = S + (long)b * ss;
  C acc[QB];
#pragma unroll
  for (int c = 0; c < QB; ++c) acc[c] = cmake<C>((T)0, (T)0);
  for (int i = 0; i < p; ++i) {
    const C sv = Sb[(long)i * L + l];
#pragma unroll
    for (int c = 0; c < QB; ++c) {
      const C cv = Cs[i][c];
      acc[c].x = fma(sv.x, cv.x, fma(-sv.y, cv.y, acc[c].x));
      acc[c].y = fma(sv.x, cv.y, fma(sv.y, cv.x, acc[c].y));
    }
  }
  C *Yb = Y + (long)b * sy;
  const float2 *Zb = Z ? Z + (long)b * sz : nullptr;
#pragma unroll
  for (int c = 0; c < QB; ++c)
    if (j0 + c < q) {
      C v = acc[c];
      if (Zb) {
        const float2 z = Zb[(long)(j0 + c) * L + l];
        v.x += (T)z.x;
        v.y += (T)z.y;
      }
      Yb[(long)(j0 + c) * L + l] = v;
    }
}

template <typename T, int QB>
static void block_update_t(int nb, long L, int p, int q, const void *S, long ss, const void *C, long sc, void *Y,
                           long sy, cudaStream_t st, const int *act, const void *Z, long sz) {
  const dim3 grid((unsigned)((L + 255) / 256), (unsigned)((q + QB - 1) / QB), nb);
  block_update_kernel<T, QB><<<grid, 256, 0, st>>>(static_cast<const cplx<T> *>(S), ss,
                                                   static_cast<const double2 *>(C), sc, static_cast<cplx<T> *>(Y), sy,
                                                   static_cast<const float2 *>(Z), sz, L, p, q, act);
}

// the column-group width for q outputs among `widths`: fewest idle columns, then fewest groups
static int update_width(int q, std::initializer_list<int> widths) {
  int best = 0;
  for (int w : widths) {
    if (best == 0) {
      best = w;
      continue;
    }
    const int idle = (q + w - 1) / w * w - q, best_idle = (q + best - 1) / best * best - q;
    if (idle < best_idle || (idle == best_idle && (q + w - 1) / w < (q + best - 1) / best)) best = w;
  }
  return best;
}

int launch_block_update(int nb, long L, int p, int q, int dtype, const void *S, long ss, const void *C, long sc,
                        void *Y, long sy, cudaStream_t st, const int *act, const void *Z, long sz) {
  if (nb == 0 || q == 0) return PC_OK;
  if (p > UPD_PMAX) {
    set_error("block_update: at most 64 input columns");
    return PC_EINVAL;
  }
  if (dtype == PC_C128) {
    if (update_width(q, {8, 16}) == 8)
      block_update_t<double, 8>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz);
    else
      block_update_t<double, 16>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz);
  } else {
    switch (update_width(q, {8, 10, 12, 16, 20, 24})) {
      case 8: block_update_t<float, 8>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz); break;
      case 10: block_update_t<float, 10>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz); break;
      case 12: block_update_t<float, 12>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz); break;
      case 16: block_update_t<float, 16>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz); break;
      case 20: block_update_t<float, 20>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz); break;
      default: block_update_t<float, 24>(nb, L, p, q, S, ss, C, sc, Y, sy, st, act, Z, sz); break;
    }
  }
  PC_CK_LAUNCH();
  return PC_OK;
}

// ------------------------------------------------------------------------------------------------ initial block input
// complex64 -> complex128 copy of the first q columns (q L entries) of k-points b0 + blockIdx.y
__global__ void __launch_bounds__(256) copy_x0_kernel(const float2 *__restrict__ X0, long qL, int b0,
                                                      double2 *__restrict__ X, long sx) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= qL) return;
  const long b = b0 + blockIdx.y;
  const float2 v = X0[b * qL + i];
  X[b * sx + i] = make_double2((double)v.x, (double)v.y);
}

int launch_copy_x0(const pc_ctx *ctx, int b0, int nbk, int dtype, void *X, long sx, cudaStream_t st) {
  if (!ctx->x0 || nbk == 0 || ctx->x0n == 0) return PC_OK;
  const long qL = (long)ctx->x0n * 3 * ctx->n;
  if (ctx->x0_c128) {
    // complex128 blocks (the FP64 finish) into complex128 panels only
    if (dtype != PC_C128) {
      set_error("copy_x0: a complex128 initial block needs complex128 panels");
      return PC_EINVAL;
    }
    const double2 *src = static_cast<const double2 *>(ctx->x0);
    PC_CK(cudaMemcpy2DAsync(static_cast<double2 *>(X) + (long)b0 * sx, sizeof(double2) * sx, src + (long)b0 * qL,
                            sizeof(double2) * qL, sizeof(double2) * qL, nbk, cudaMemcpyDeviceToDevice, st));
    return PC_OK;
  }
  const float2 *src = static_cast<const float2 *>(ctx->x0);
  if (dtype == PC_C64) {
    // one strided copy: nbk rows of qL complex64 entries, source pitch qL, destination pitch sx
    PC_CK(cudaMemcpy2DAsync(static_cast<float2 *>(X) + (long)b0 * sx, sizeof(float2) * sx, src + (long)b0 * qL,
                            sizeof(float2) * qL, sizeof(float2) * qL, nbk, cudaMemcpyDeviceToDevice, st));
    return PC_OK;
  }
  copy_x0_kernel<<<dim3((unsigned)((qL + 255) / 256), nbk), 256, 0, st>>>(src, qL, b0, static_cast<double2 *>(X), sx);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ------------------------------------------------------------------------------------------------ residual
__global__ void __launch_bounds__(256) residual_partial_kernel(const double2 *__restrict__ X, long sx,
                                                              const double2 *__restrict__ AX, long sax,
                                                              const double *__restrict__ theta,
                                                              double2 *__restrict__ R, long sr, long L, long chunk,
                                                              int m, double *__restrict__ part,
                                                              const int *__restrict__ act) {
  const int bi = blockIdx.z, j = blockIdx.y;
  const int b = act ? act[bi] : bi;
  const double th = theta[(long)b * m + j];
  const double2 *x = X + (long)b * sx + (long)j * L;
  const double2 *ax = AX + (long)b * sax + (long)j * L;
  double2 *rr = R + (long)b * sr + (long)j * L;
  double sr2 = 0.0, sx2 = 0.0;
  const long beg = (long)blockIdx.x * chunk, end = min(L, beg + chunk);
  for (long l = beg + threadIdx.x; l < end; l += blockDim.x) {
    const double2 xv = x[l], av = ax[l];
    const double2 rv = cmake<double2>(av.x - th * xv.x, av.y - th * xv.y);
    rr[l] = rv;
    sr2 += rv.x * rv.x + rv.y * rv.y;
    sx2 += xv.x * xv.x + xv.y * xv.y;
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = sr2;
  red[1][threadIdx.x] = sx2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double *o = part + (((long)bi * m + j) * gridDim.x + blockIdx.x) * 2;
    o[0] = red[0][0];
    o[1] = red[1][0];
  }
}

__global__ void residual_reduce_kernel(const double *__restrict__ part, int nchunk, int m,
                                       const int *__restrict__ act, double *__restrict__ norms) {
  const int bi = blockIdx.x;
  const int b = act ? act[bi] : bi;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s0 = 0, s1 = 0;
    for (int c = 0; c < nchunk; ++c) {
      s0 += part[(((long)bi * m + j) * nchunk + c) * 2];
      s1 += part[(((long)bi * m + j) * nchunk + c) * 2 + 1];
    }
    norms[((long)b * m + j) * 2] = sqrt(s0);
    norms[((long)b * m + j) * 2 + 1] = sqrt(s1);
  }
}

void launch_residual_reduce(int nb, int nchunk, int m, const double *part, const int *act, double *norms,
                            cudaStream_t st) {
  residual_reduce_kernel<<<nb, 64, 0, st>>>(part, nchunk, m, act, norms);
}

static int residual_chunks(long L) { return (int)std::min<long>(32, std::max<long>(1, L / 4096)); }

size_t residual_scratch_bytes(int nb, long L, int m) {
  return sizeof(double) * 2 * (size_t)nb * m * residual_chunks(L);
}

int launch_residual(int nb, long L, int m, const void *X, long sx, const void *AX, long sax, const double *theta,
                    void *R, long sr, double *norms, void *scratch, size_t scratch_bytes, cudaStream_t st,
                    const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  const int nchunk = residual_chunks(L);
  if (residual_scratch_bytes(nb, L, m) > scratch_bytes) {
    set_error("residual: scratch too small");
    return PC_EINVAL;
  }
  const long chunk = (L + nchunk - 1) / nchunk;
  residual_partial_kernel<<<dim3(nchunk, m, nb), 256, 0, st>>>(
      static_cast<const double2 *>(X), sx, static_cast<const double2 *>(AX), sax, theta, static_cast<double2 *>(R),
      sr, L, chunk, m, static_cast<double *>(scratch), act);
  PC_CK_LAUNCH();
  residual_reduce_kernel<<<nb, 64, 0, st>>>(static_cast<double *>(scratch), nchunk, m, act, norms);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ------------------------------------------------------------------------------------------------ mixed precision
// Residual for the mixed-precision solve: r = AX - theta x in the precision TX of the block (FP64 once X is held in
// FP64, complex64 before), stored as complex64 twice (the preconditioner input slot and the copy kept for the
// Rayleigh-Ritz coupling R^H Q); optionally also complex64 copies of X and AX for the complex64 Gram products.
// Column sums |r|^2, |x|^2 accumulate per thread in TX and per block in FP64.
template <typename TX>
__global__ void __launch_bounds__(256) residual_mixed_partial_kernel(
    const cplx<TX> *__restrict__ X, long sx, const cplx<TX> *__restrict__ AX, long sax, const double *__restrict__ theta,
    float2 *__restrict__ R1, long sr1, float2 *__restrict__ R2, long sr2, float2 *__restrict__ X32, long sx32,
    float2 *__restrict__ AX32, long sax32, long L, long chunk, int m, double *__restrict__ part,
    const int *__restrict__ act) {
  const int bi = blockIdx.z, j = blockIdx.y;
  const int b = act ? act[bi] : bi;
  const TX th = (TX)theta[(long)b * m + j];
  const cplx<TX> *x = X + (long)b * sx + (long)j * L;
  const cplx<TX> *ax = AX + (long)b * sax + (long)j * L;
  float2 *r1 = R1 + (long)b * sr1 + (long)j * L;
  float2 *r2 = R2 + (long)b * sr2 + (long)j * L;
  float2 *x32 = X32 ? X32 + (long)b * sx32 + (long)j * L : nullptr;
  float2 *ax32 = AX32 ? AX32 + (long)b * sax32 + (long)j * L : nullptr;
  float sr = 0.f, sxx = 0.f;  // column sums need ~3 digits: FP32 per thread, FP64 per block
  const long beg = (long)blockIdx.x * chunk, end = min(L, beg + chunk);
  for (long l = beg + threadIdx.x; l < end; l += blockDim.x) {
    const cplx<TX> xv = x[l], av = ax[l];
    float rx, ry;
    if constexpr (std::is_same<TX, double>::value) {
      // r = ax - theta x cancels to ~tol |ax|: double-float arithmetic keeps it exact to ~2^-44 |ax| on the FP32 pipe
      const df t = df_from((double)th);
      const df rxd = df_sub(df_from(av.x), df_mul(t, df_from(xv.x)));
      const df ryd = df_sub(df_from(av.y), df_mul(t, df_from(xv.y)));
      rx = rxd.hi + rxd.lo;
      ry = ryd.hi + ryd.lo;
    } else {
      rx = av.x - th * xv.x;
      ry = av.y - th * xv.y;
    }
    const float2 rf = make_float2(rx, ry);
    r1[l] = rf;
    r2[l] = rf;
    if (x32) {
      x32[l] = make_float2((float)xv.x, (float)xv.y);
      ax32[l] = make_float2((float)av.x, (float)av.y);
    }
    sr += rx * rx + ry * ry;
    sxx += (float)xv.x * (float)xv.x + (float)xv.y * (float)xv.y;
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = (double)sr;
  red[1][threadIdx.x] = (double)sxx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double *o = part + (((long)bi * m + j) * gridDim.x + blockIdx.x) * 2;
    o[0] = red[0][0];
    o[1] = red[1][0];
  }
}

int launch_residual_mixed(int nb, long L, int m, int dtype_x, const void *X, long sx, const void *AX, long sax,
                          const double *theta, void *R1, long sr1, void *R2, long sr2, void *X32, long sx32,
                          void *AX32, long sax32, double *norms, void *scratch, size_t scratch_bytes,
                          cudaStream_t st, const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  const int nchunk = residual_chunks(L);
  if (residual_scratch_bytes(nb, L, m) > scratch_bytes) {
    set_error("residual_mixed: scratch too small");
    return PC_EINVAL;
  }
  const long chunk = (L + nchunk - 1) / nchunk;
  double *part = static_cast<double *>(scratch);
  dim3 grid(nchunk, m, nb);
  if (dtype_x == PC_C128)
    residual_mixed_partial_kernel<double><<<grid, 256, 0, st>>>(
        static_cast<const double2 *>(X), sx, static_cast<const double2 *>(AX), sax, theta, static_cast<float2 *>(R1),
        sr1, static_cast<float2 *>(R2), sr2, static_cast<float2 *>(X32), sx32, static_cast<float2 *>(AX32), sax32, L,
        chunk, m, part, act);
  else
    residual_mixed_partial_kernel<float><<<grid, 256, 0, st>>>(
        static_cast<const float2 *>(X), sx, static_cast<const float2 *>(AX), sax, theta, static_cast<float2 *>(R1),
        sr1, static_cast<float2 *>(R2), sr2, static_cast<float2 *>(X32), sx32, static_cast<float2 *>(AX32), sax32, L,
        chunk, m, part, act);
  PC_CK_LAUNCH();
  residual_reduce_kernel<<<nb, 64, 0, st>>>(part, nchunk, m, act, norms);
  PC_CK_LAUNCH();
  return PC_OK;
}

// Completes the Rayleigh-Ritz pencil of the mixed solve (n = m + nq columns [X | Q]) from RS = R^H [X | Q]
// ([nb][m][n]) and AX = X Theta + R (Op Hermitian), so that no product multiplies X by the large AQ in complex64:
//   H[i][m+j] = theta_i G[i][m+j] + (R^H Q)[i][j], mirrored;
// and, for k-points whose block X is held in FP64 (phase[b] == 2), G[:m,:m] = GX (the FP64 X^H X) and
//   H[:m,:m] = the Hermitian part of (theta_i GX[i][j] + (R^H X)[i][j]).
__global__ void rr_patch_kernel(double2 *__restrict__ G, double2 *__restrict__ H, int n, int m,
                                const double2 *__restrict__ RS, const double *__restrict__ theta,
                                const double2 *__restrict__ GX, const int *__restrict__ phase,
                                const int *__restrict__ act, long sg, long srs) {
  const int b = act ? act[blockIdx.x] : (int)blockIdx.x;
  double2 *Gb = G + (long)b * sg, *Hb = H + (long)b * sg;
  const double2 *RSb = RS + (long)b * srs;
  const double *th = theta + (long)b * m;
  const int nq = n - m;
  for (int e = threadIdx.x; e < m * nq; e += blockDim.x) {
    const int i = e / nq, j = e - i * nq;
    const double2 g = Gb[i * n + m + j], rq = RSb[i * n + m + j];
    const double2 h = cmake<double2>(th[i] * g.x + rq.x, th[i] * g.y + rq.y);
    Hb[i * n + m + j] = h;
    Hb[(m + j) * n + i] = cmake<double2>(h.x, -h.y);
  }
  if (phase && phase[b] == 2) {
    const double2 *GXb = GX + (long)b * m * m;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e - i * m;
      const double2 gij = GXb[i * m + j], gji = GXb[j * m + i];
      const double2 rij = RSb[i * n + j], rji = RSb[j * n + i];
      // M = Theta GX + R^H X; H = (M + M^H) / 2
      const double2 mij = cmake<double2>(th[i] * gij.x + rij.x, th[i] * gij.y + rij.y);
      const double2 mji = cmake<double2>(th[j] * gji.x + rji.x, th[j] * gji.y + rji.y);
      Gb[i * n + j] = gij;
      Hb[i * n + j] = cmake<double2>(0.5 * (mij.x + mji.x), 0.5 * (mij.y - mji.y));
    }
  }
}

int launch_rr_patch(int nb, int n, int m, void *G, void *H, const void *RS, const double *theta, const void *GX,
                    const int *phase, cudaStream_t st, const int *act, long sg, long srs) {
  if (nb == 0) return PC_OK;
  rr_patch_kernel<<<nb, 256, 0, st>>>(static_cast<double2 *>(G), static_cast<double2 *>(H), n, m,
                                      static_cast<const double2 *>(RS), theta, static_cast<const double2 *>(GX),
                                      phase, act, sg > 0 ? sg : (long)n * n, srs > 0 ? srs : (long)m * n);
  PC_CK_LAUNCH();
  return PC_OK;
}

// Y (double-float pairs, PC_DFS) = X (complex64) for m columns of length L per k-point: (x, 0) is exact.
__global__ void widen_kernel(const float2 *__restrict__ X, long sx, float4 *__restrict__ Y, long sy, long L,
                             const int *__restrict__ act) {
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z, j = blockIdx.y;
  const float2 *x = X + (long)b * sx + (long)j * L;
  float4 *y = Y + (long)b * sy + (long)j * L;
  for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (long)gridDim.x * blockDim.x) {
    const float2 v = x[l];
    y[l] = make_float4(v.x, 0.f, v.y, 0.f);
  }
}

int launch_widen(int nb, long L, int m, const void *X, long sx, void *Y, long sy, cudaStream_t st, const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  const unsigned gx = (unsigned)std::min<long>(256, (L + 255) / 256);
  widen_kernel<<<dim3(gx, m, nb), 256, 0, st>>>(static_cast<const float2 *>(X), sx, static_cast<float4 *>(Y), sy, L,
                                                act);
  PC_CK_LAUNCH();
  return PC_OK;
}

// Y (complex128) = hi + lo of X (double-float pairs) for m columns of length L per k-point.
__global__ void pairs_to_c128_kernel(const float4 *__restrict__ X, long sx, double2 *__restrict__ Y, long sy, long L,
                                     const int *__restrict__ act) {
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z, j = blockIdx.y;
  const float4 *x = X + (long)b * sx + (long)j * L;
  double2 *y = Y + (long)b * sy + (long)j * L;
  for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (long)gridDim.x * blockDim.x)
    y[l] = ld_c128(x + l);
}

int launch_pairs_to_c128(int nb, long L, int m, const void *X, long sx, void *Y, long sy, cudaStream_t st,
                         const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  const unsigned gx = (unsigned)std::min<long>(256, (L + 255) / 256);
  pairs_to_c128_kernel<<<dim3(gx, m, nb), 256, 0, st>>>(static_cast<const float4 *>(X), sx, static_cast<double2 *>(Y),
                                                        sy, L, act);
  PC_CK_LAUNCH();
  return PC_OK;
}


// ------------------------------------------------------------------------------------------------ k = 0 projection
// Removes the mean of each component of each column for k-points with flags[b] != 0 (the constant kernel fields).
// Two launches, DEFL_SPLIT blocks per (column, component) each: partial sums over a slice of the component (FP64,
// from FP32 per-thread sums for complex64 data), then every block adds the slices' partial sums and subtracts the
// mean from its own slice. Blocks of k-points without the flag return at once, so a launch can cover a whole active
// list. S: the element storage, float2 (complex64), double2 (complex128) or float4 (double-float pairs). Scratch:
// [nb][3 m][DEFL_SPLIT] double2.
constexpr int DEFL_SPLIT = 16;

template <typename S>
__global__ void __launch_bounds__(256) deflate_sum_kernel(const S *__restrict__ X, long sx, long n,
                                                         const int *__restrict__ flags, const int *__restrict__ act,
                                                         double2 *__restrict__ part) {
  const int bi = blockIdx.y, col = blockIdx.x / DEFL_SPLIT, sl = blockIdx.x % DEFL_SPLIT;  // col = j * 3 + comp
  const int b = act ? act[bi] : bi;
  if (!flags[b]) return;
  const long len = (n + DEFL_SPLIT - 1) / DEFL_SPLIT, l0 = sl * len, l1 = min(n, l0 + len);
  const S *x = X + (long)b * sx + (long)col * n;
  double sr = 0.0, si = 0.0;
  if constexpr (std::is_same<S, float2>::value) {
    // complex64 data: per-thread sums in FP32 (their rounding is that of the data), FP64 from the warp sums on
    float fr = 0.f, fi = 0.f;
    for (long l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
      const float2 v = x[l];
      fr += v.x;
      fi += v.y;
    }
    sr = fr;
    si = fi;
  } else {
    for (long l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
      const double2 v = ld_c128(x + l);
      sr += v.x;
      si += v.y;
    }
  }
  __shared__ double red[2][8];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = sr;
    red[1][w] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mr = 0.0, mi = 0.0;
    for (int i = 0; i < nw; ++i) {
      mr += red[0][i];
      mi += red[1][i];
    }
    part[((long)bi * gridDim.x + blockIdx.x)] = make_double2(mr, mi);
  }
}

template <typename S>
__global__ void __launch_bounds__(256) deflate_sub_kernel(S *__restrict__ X, long sx, long n,
                                                         const int *__restrict__ flags, const int *__restrict__ act,
                                                         const double2 *__restrict__ part) {
  const int bi = blockIdx.y, col = blockIdx.x / DEFL_SPLIT, sl = blockIdx.x % DEFL_SPLIT;
  const int b = act ? act[bi] : bi;
  if (!flags[b]) return;
  double mr = 0.0, mi = 0.0;
  const double2 *pc = part + (long)bi * gridDim.x + (long)col * DEFL_SPLIT;
  for (int i = 0; i < DEFL_SPLIT; ++i) {
    mr += pc[i].x;
    mi += pc[i].y;
  }
  mr /= (double)n;
  mi /= (double)n;
  const long len = (n + DEFL_SPLIT - 1) / DEFL_SPLIT, l0 = sl * len, l1 = min(n, l0 + len);
  S *x = X + (long)b * sx + (long)col * n;
  if constexpr (std::is_same<S, float4>::value) {
    const df dr = df_from(mr), di = df_from(mi);
    for (long l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
      cdf v = ld_cdf(x + l);
      v.re = df_sub(v.re, dr);
      v.im = df_sub(v.im, di);
      st_cdf(x + l, v);
    }
  } else {
    using T = decltype(S{}.x);
    const T tr = (T)mr, ti = (T)mi;
    for (long l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
      x[l].x -= tr;
      x[l].y -= ti;
    }
  }
}

template <typename S>
static void deflate_t(int nb, long n, int m, S *X, long sx, const int *flags, double2 *part, cudaStream_t st,
                      const int *act) {
  const dim3 grid(3 * m * DEFL_SPLIT, nb);
  deflate_sum_kernel<S><<<grid, 256, 0, st>>>(X, sx, n, flags, act, part);
  deflate_sub_kernel<S><<<grid, 256, 0, st>>>(X, sx, n, flags, act, part);
}

size_t deflate_scratch_bytes(int nb, int m) { return sizeof(double2) * (size_t)nb * 3 * m * DEFL_SPLIT; }

int launch_deflate(int nb, long n, int m, void *X, long sx, const int *flags, void *scratch, cudaStream_t st,
                   const int *act, int dtype) {
  if (nb == 0 || m == 0) return PC_OK;
  double2 *part = static_cast<double2 *>(scratch);
  if (dtype == PC_C128)
    deflate_t<double2>(nb, n, m, static_cast<double2 *>(X), sx, flags, part, st, act);
  else if (dtype == PC_DFS)
    deflate_t<float4>(nb, n, m, static_cast<float4 *>(X), sx, flags, part, st, act);
  else
    deflate_t<float2>(nb, n, m, static_cast<float2 *>(X), sx, flags, part, st, act);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ------------------------------------------------------------------------------------------------ initial blocks
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return z;
}

template <typename S>
__global__ void init_block_kernel(S *__restrict__ X, long sx, long L, uint64_t seed, int kidx0,
                                  const int *__restrict__ mask, int m, const int *__restrict__ act) {
  const uint64_t G = 0x9E3779B97F4A7C15ULL;
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z, j = blockIdx.y;
  if (mask && !mask[b * m + j]) return;
  const uint64_t stream = (uint64_t)(kidx0 + b) * 4096ULL + (uint64_t)j;
  const uint64_t key = mix64(seed + G * (stream + 1ULL));
  S *x = X + (long)b * sx + (long)j * L;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += (long)gridDim.x * blockDim.x) {
    const uint64_t d1 = mix64(key + G * (2ULL * (uint64_t)e + 1ULL));
    const uint64_t d2 = mix64(key + G * (2ULL * (uint64_t)e + 2ULL));
    if constexpr (std::is_same<S, float2>::value) {
      // complex64 start block: the same counter-based uniforms (their top 24 bits) and Box-Muller in FP32
      const float u1 = ((float)(d1 >> 40) + 0.5f) * 0x1.0p-24f;
      const float u2 = ((float)(d2 >> 40) + 0.5f) * 0x1.0p-24f;
      const float rad = sqrtf(-2.0f * logf(u1));
      float s, c;
      sincospif(2.0f * u2, &s, &c);
      x[e] = make_float2(rad * c, rad * s);
      continue;
    }
    const double u1 = ((double)(d1 >> 11) + 0.5) * 0x1.0p-53;
    const double u2 = ((double)(d2 >> 11) + 0.5) * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    if constexpr (std::is_same<S, float4>::value)
      st_cdf(x + e, cdf_from(cmake<double2>(rad * c, rad * s)));
    else if constexpr (std::is_same<S, double2>::value)
      x[e] = cmake<double2>(rad * c, rad * s);
  }
}

int launch_init_block(int nb, long L, int m, uint64_t seed, int kidx0, void *X, long sx, cudaStream_t st,
                      const int *mask, const int *act, int dtype) {
  if (nb == 0 || m == 0) return PC_OK;
  const unsigned gx = (unsigned)std::min<long>(256, (L + 255) / 256);
  if (dtype == PC_DFS)
    init_block_kernel<float4><<<dim3(gx, m, nb), 256, 0, st>>>(static_cast<float4 *>(X), sx, L, seed, kidx0, mask, m,
                                                               act);
  else if (dtype == PC_C64)
    init_block_kernel<float2><<<dim3(gx, m, nb), 256, 0, st>>>(static_cast<float2 *>(X), sx, L, seed, kidx0, mask, m,
                                                               act);
  else
    init_block_kernel<double2><<<dim3(gx, m, nb), 256, 0, st>>>(static_cast<double2 *>(X), sx, L, seed, kidx0, mask,
                                                                m, act);
  PC_CK_LAUNCH();
  return PC_OK;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_gram(int nb, long L, int p, int q, int dtype, const void *A, long sa, const void *B, long sb,
                       void *G, void *stream) {
  PC_REQUIRE(A && B && G, "pc_gram: null argument");
  PC_REQUIRE(nb >= 0 && L >= 0 && p >= 0 && q >= 0 && p <= 64 && q <= 64, "pc_gram: bad sizes");
  PC_REQUIRE(dtype == PC_C128 || dtype == PC_C64, "pc_gram: bad dtype");
  DevBuf tmp;
  PC_CK(tmp.reserve(std::max<size_t>(16, gram_scratch_bytes(nb, L, p, q))));
  int rc = launch_gram(nb, L, p, q, dtype, A, sa, B, sb, G, tmp.p, tmp.bytes, (cudaStream_t)stream, nullptr);
  if (rc) return rc;
  PC_CK(cudaStreamSynchronize((cudaStream_t)stream));  // tmp is released on return
  return PC_OK;
}

extern "C" int pc_gram_pair(int nb, long L, int p, int dtype, const void *S, long ss, const void *AS, void *G,
                            void *H, void *stream) {
  PC_REQUIRE(S && AS && G && H, "pc_gram_pair: null argument");
  PC_REQUIRE(nb >= 0 && L >= 0 && p >= 1 && p <= 64, "pc_gram_pair: bad sizes");
  PC_REQUIRE(dtype == PC_C128 || dtype == PC_C64, "pc_gram_pair: bad dtype");
  DevBuf tmp;
  PC_CK(tmp.reserve(std::max<size_t>(16, gram_pair_scratch_bytes(nb, L, p))));
  int rc = launch_gram_pair(nb, L, p, dtype, S, AS, ss, G, H, tmp.p, tmp.bytes, (cudaStream_t)stream, nullptr);
  if (rc) return rc;
  PC_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return PC_OK;
}

extern "C" int pc_gram_pair_coupled(int nb, long L, int p, int q, const void *S, long ss, const void *AS,
                                    const void *R, long sr, void *G, void *H, void *RQ, void *stream) {
  PC_REQUIRE(S && AS && R && G && H && RQ, "pc_gram_pair_coupled: null argument");
  PC_REQUIRE(nb >= 0 && L >= 0 && p >= 1 && p <= 64 && q >= 1 && q <= 64, "pc_gram_pair_coupled: bad sizes");
  DevBuf tmp;
  PC_CK(tmp.reserve(std::max<size_t>(16, gram_pair_coupled_scratch_bytes(nb, L, p, q))));
  int rc = launch_gram_pair_coupled(nb, L, p, q, PC_C64, S, AS, ss, R, sr, G, H, RQ, tmp.p, tmp.bytes,
                                    (cudaStream_t)stream, nullptr);
  if (rc) return rc;
  PC_CK(cudaStreamSynchronize((cudaStream_t)stream));  // tmp is released on return
  return PC_OK;
}

extern "C" int pc_block_update(int nb, long L, int p, int q, int dtype, const void *S, long ss, const void *C, void *Y,
                               long sy, void *stream) {
  PC_REQUIRE(S && C && Y, "pc_block_update: null argument");
  PC_REQUIRE(nb >= 0 && L >= 0 && p >= 0 && q >= 0 && p <= 64 && q <= 64, "pc_block_update: bad sizes");
  PC_REQUIRE(dtype == PC_C128 || dtype == PC_C64, "pc_block_update: bad dtype");
  return launch_block_update(nb, L, p, q, dtype, S, ss, C, (long)p * q, Y, sy, (cudaStream_t)stream, nullptr);
}

extern "C" int pc_residual(int nb, long L, int m, const void *X, const void *AX, const double *theta, void *R,
                           double *norms, void *stream) {
  PC_REQUIRE(X && AX && theta && R && norms, "pc_residual: null argument");
  PC_REQUIRE(nb >= 0 && L >= 0 && m >= 0 && m <= 64, "pc_residual: bad sizes");
  DevBuf tmp;
  PC_CK(tmp.reserve(std::max<size_t>(16, residual_scratch_bytes(nb, L, m))));
  const long blk = (long)m * L;
  int rc = launch_residual(nb, L, m, X, blk, AX, blk, theta, R, blk, norms, tmp.p, tmp.bytes, (cudaStream_t)stream,
                           nullptr);
  if (rc) return rc;
  PC_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return PC_OK;
}

extern "C" int pc_init_block(int nb, long L, int m, uint64_t seed, int kidx0, void *X, void *stream) {
  PC_REQUIRE(X, "pc_init_block: null argument");
  PC_REQUIRE(nb >= 0 && L >= 0 && m >= 0 && m < 4096, "pc_init_block: bad sizes");
  return launch_init_block(nb, L, m, seed, kidx0, X, (long)m * L, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------------------------------ no-allocation
// pc_gram_pair_noalloc: the Gram pair of pc_gram_pair for callers that must not allocate device memory. Its
// per-chunk partial sums live in this fixed array instead of a cudaMalloc'd buffer. The array is part of the
// library image, so every GPU that loads the library holds these bytes until the process exits.
namespace pc {

constexpr size_t NOALLOC_SCRATCH_BYTES = 4u << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device. In host code the symbol names a host-side
// stand-in, not device memory, so kernels must be given the address returned by cudaGetSymbolAddress.
static int noalloc_scratch_address(void **out) {
  static std::mutex mu;
  static void *addr[64] = {};
  int dev = 0;
  PC_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("pc_gram_pair_noalloc: device index %d out of range", dev);
    return PC_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    PC_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = p;
  }
  *out = addr[dev];
  return PC_OK;
}

}  // namespace pc

extern "C" int pc_gram_pair_noalloc(int nb, long L, int p, int dtype, const void *S, long ss, const void *AS, void *G,
                                    void *H, void *stream) {
  PC_REQUIRE(S && AS && G && H, "pc_gram_pair_noalloc: null argument");
  PC_REQUIRE(nb >= 0 && L >= 0 && p >= 1 && p <= 64, "pc_gram_pair_noalloc: bad sizes");
  PC_REQUIRE(dtype == PC_C128 || dtype == PC_C64, "pc_gram_pair_noalloc: bad dtype");
  if (nb == 0) return PC_OK;
  // two partial panels (G and H) of nb * nchunk * p * p complex128 must fit in the fixed array
  const size_t per_chunk = 2 * sizeof(double2) * (size_t)nb * p * p;
  const size_t fit = NOALLOC_SCRATCH_BYTES / per_chunk;
  if (fit < 1) {
    set_error("pc_gram_pair_noalloc: nb * p * p = %zu exceeds the fixed scratch (at most %zu, i.e. 2*16*nb*p*p <= %zu "
              "bytes)", (size_t)nb * p * p, NOALLOC_SCRATCH_BYTES / (2 * sizeof(double2)), NOALLOC_SCRATCH_BYTES);
    return PC_EINVAL;
  }
  void *scratch = nullptr;
  int rc = noalloc_scratch_address(&scratch);
  if (rc) return rc;
  const int nchunk = (int)std::min<size_t>((size_t)gram_chunks(nb, L), fit);
  long chunk = (L + nchunk - 1) / nchunk;
  chunk = (chunk + GRAM_TL - 1) / GRAM_TL * GRAM_TL;
  double2 *part = static_cast<double2 *>(scratch);
  cudaStream_t st = (cudaStream_t)stream;
  // every partial entry the reduction reads (i <= j of each chunk) is written first in this call: nothing to clear
  rc = dtype == PC_C128 ? launch_gram_pair_t<double>(nb, L, p, S, AS, ss, part, nchunk, chunk, st, nullptr)
                        : launch_gram_pair_t<float>(nb, L, p, S, AS, ss, part, nchunk, chunk, st, nullptr);
  if (rc) return rc;
  gram_pair_reduce_kernel<<<dim3(nb, (p * p + 255) / 256), 256, 0, st>>>(
      part, part + (size_t)nb * nchunk * p * p, nchunk, p, nullptr, static_cast<double2 *>(G),
      static_cast<double2 *>(H), (long)p * p);
  PC_CK_LAUNCH();
  return PC_OK;
}
