// The FP64-accurate kernels of the mixed-precision solve, in double-float arithmetic (dfloat.cuh): the block X and
// its image AX stay FP64 in memory, every element is split into hi + lo FP32 on load, and all arithmetic runs on
// the FP32 pipe (GB300: 75 TFLOP/s FP32 against 1.2 TFLOP/s FP64).
//   op_df_kernel      AX = Op X  (the stencil of stencil.cu; differences, shifts, M0, gamma in double-float)
//   update_df_kernel  X' = X C + Z  (Z: the complex64 correction [W P] coef_{W,P})
//   gram_df_kernel    G = X^H X, H = X^H AX  (upper triangles, Hermitian mirrors)
//   resid_df_kernel   R = AX - X Theta -> complex64 copies, plus complex64 copies of X and AX, and column norms
#include <cmath>

#include "dfloat.cuh"
#include "pc_internal.cuh"

namespace pc {

// ---------------------------------------------------------------- stencil
// (D f)_r = ih (f_{r+1} - f_r) + i kh (f_r + f_{r+1});  (D' g)_r = ih (g_{r-1} - g_r) - i kh (g_{r-1} + g_r)
__device__ __forceinline__ cdf dfwd_df(cdf f0, cdf f1, float ih, df kh) {
  const cdf a = cdf_sub(f1, f0), s = cdf_add(f0, f1);
  // ih a + i kh s = (ih a.re - kh s.im) + i (ih a.im + kh s.re)
  return cdf{df_sub(df_scale2(a.re, ih), df_mul(kh, s.im)), df_add(df_scale2(a.im, ih), df_mul(kh, s.re))};
}
__device__ __forceinline__ cdf dbwd_df(cdf gm, cdf g0, float ih, df kh) {
  const cdf a = cdf_sub(gm, g0), s = cdf_add(gm, g0);
  // ih a - i kh s = (ih a.re + kh s.im) + i (ih a.im - kh s.re)
  return cdf{df_add(df_scale2(a.re, ih), df_mul(kh, s.im)), df_sub(df_scale2(a.im, ih), df_mul(kh, s.re))};
}

template <int TX, int TY, int TZ> constexpr size_t op_df_smem_bytes() {
  return sizeof(cdf) * (size_t)(3 * (TZ + 2) * (TY + 2) * (TX + 2) + 3 * (TZ + 1) * (TY + 1) * (TX + 1) +
                                (TZ + 1) * (TY + 1) * (TX + 1));
}

// Same tiling as op_kernel (stencil.cu): a face tile with a one-point halo, e = M0 A' v on the tile grown upward,
// c = B v on the tile grown downward, then y = A e + gamma B' c. The grid spacing factor ih = N is a power of two,
// so scaling by it is exact in double-float.
template <int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) op_df_kernel(const double2 *__restrict__ X, long sx, double2 *__restrict__ Y,
                                                    long sy, const double *__restrict__ m0,
                                                    const KParam *__restrict__ kp, const int *__restrict__ act,
                                                    int logN) {
  constexpr int VX = TX + 2, VY = TY + 2, VZ = TZ + 2;
  constexpr int EX = TX + 1, EY = TY + 1, EZ = TZ + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cdf *v = reinterpret_cast<cdf *>(smem_raw);
  cdf *e = v + 3 * VZ * VY * VX;
  cdf *c = e + 3 * EZ * EY * EX;
  const int N = 1 << logN, mask = N - 1;
  const long n = 1L << (3 * logN);
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int j = blockIdx.y;
  const int tilesX = N / TX, tilesY = N / TY;
  int t = blockIdx.x;
  const int x0 = (t % tilesX) * TX;
  t /= tilesX;
  const int y0 = (t % tilesY) * TY;
  const int z0 = (t / tilesY) * TZ;
  const double2 *Xb = X + (long)b * sx + (long)j * 3 * n;
  double2 *Yb = Y + (long)b * sy + (long)j * 3 * n;
  const KParam p = kp[b];
  const df kh0 = df_from(0.5 * p.k[0]), kh1 = df_from(0.5 * p.k[1]), kh2 = df_from(0.5 * p.k[2]);
  const df gam = df_from(p.gamma);
  const float ih = (float)N;

  for (int i = threadIdx.x; i < 3 * VZ * VY * VX; i += blockDim.x) {
    int lx = i % VX, r = i / VX;
    int ly = r % VY;
    r /= VY;
    int lz = r % VZ, comp = r / VZ;
    int gx = (x0 + lx - 1) & mask, gy = (y0 + ly - 1) & mask, gz = (z0 + lz - 1) & mask;
    v[i] = cdf_from(Xb[comp * n + ((long)gz << (2 * logN)) + ((long)gy << logN) + gx]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < EZ * EY * EX; i += blockDim.x) {
    const int ex = i % EX, ey = (i / EX) % EY, ez = i / (EX * EY);
#define VV(comp, dz, dy, dx) v[(((comp) * VZ + ez + 1 + (dz)) * VY + ey + 1 + (dy)) * VX + ex + 1 + (dx)]
    const cdf v1 = VV(0, 0, 0, 0), v2 = VV(1, 0, 0, 0), v3 = VV(2, 0, 0, 0);
    const cdf d3v2 = dbwd_df(VV(1, -1, 0, 0), v2, ih, kh2);
    const cdf d2v3 = dbwd_df(VV(2, 0, -1, 0), v3, ih, kh1);
    const cdf d3v1 = dbwd_df(VV(0, -1, 0, 0), v1, ih, kh2);
    const cdf d1v3 = dbwd_df(VV(2, 0, 0, -1), v3, ih, kh0);
    const cdf d2v1 = dbwd_df(VV(0, 0, -1, 0), v1, ih, kh1);
    const cdf d1v2 = dbwd_df(VV(1, 0, 0, -1), v2, ih, kh0);
#undef VV
    const int gx = (x0 + ex) & mask, gy = (y0 + ey) & mask, gz = (z0 + ez) & mask;
    const long gi = ((long)gz << (2 * logN)) + ((long)gy << logN) + gx;
    const int eo = (ez * EY + ey) * EX + ex;
    e[eo] = cdf_scale(cdf_sub(d3v2, d2v3), df_from(m0[gi]));
    e[EZ * EY * EX + eo] = cdf_scale(cdf_sub(d1v3, d3v1), df_from(m0[n + gi]));
    e[2 * EZ * EY * EX + eo] = cdf_scale(cdf_sub(d2v1, d1v2), df_from(m0[2 * n + gi]));
#define WW(comp, dz, dy, dx) v[(((comp) * VZ + ez + (dz)) * VY + ey + (dy)) * VX + ex + (dx)]
    cdf cc = dfwd_df(WW(0, 0, 0, 0), WW(0, 0, 0, 1), ih, kh0);
    cc = cdf_add(cc, dfwd_df(WW(1, 0, 0, 0), WW(1, 0, 1, 0), ih, kh1));
    cc = cdf_add(cc, dfwd_df(WW(2, 0, 0, 0), WW(2, 1, 0, 0), ih, kh2));
#undef WW
    c[eo] = cc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TZ * TY * TX; i += blockDim.x) {
    const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
#define EE(comp, dz, dy, dx) e[(((comp) * EZ + lz + (dz)) * EY + ly + (dy)) * EX + lx + (dx)]
#define CC(dz, dy, dx) c[((lz + 1 + (dz)) * EY + ly + 1 + (dy)) * EX + lx + 1 + (dx)]
    const cdf c0 = CC(0, 0, 0);
    const cdf e1 = EE(0, 0, 0, 0), e2 = EE(1, 0, 0, 0), e3 = EE(2, 0, 0, 0);
    cdf y1 = cdf_sub(dfwd_df(e3, EE(2, 0, 1, 0), ih, kh1), dfwd_df(e2, EE(1, 1, 0, 0), ih, kh2));
    y1 = cdf_add(y1, cdf_scale(dbwd_df(CC(0, 0, -1), c0, ih, kh0), gam));
    cdf y2 = cdf_sub(dfwd_df(e1, EE(0, 1, 0, 0), ih, kh2), dfwd_df(e3, EE(2, 0, 0, 1), ih, kh0));
    y2 = cdf_add(y2, cdf_scale(dbwd_df(CC(0, -1, 0), c0, ih, kh1), gam));
    cdf y3 = cdf_sub(dfwd_df(e2, EE(1, 0, 0, 1), ih, kh0), dfwd_df(e1, EE(0, 0, 1, 0), ih, kh1));
    y3 = cdf_add(y3, cdf_scale(dbwd_df(CC(-1, 0, 0), c0, ih, kh2), gam));
#undef EE
#undef CC
    const long gi = ((long)(z0 + lz) << (2 * logN)) + ((long)(y0 + ly) << logN) + x0 + lx;
    Yb[gi] = cdf_to(y1);
    Yb[n + gi] = cdf_to(y2);
    Yb[2 * n + gi] = cdf_to(y3);
  }
}

template <int TX, int TY, int TZ>
static int launch_op_df_t(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act) {
  constexpr size_t smem = op_df_smem_bytes<TX, TY, TZ>();
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(op_df_kernel<TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  const int N = ctx->N;
  dim3 grid((N / TX) * (N / TY) * (N / TZ), m, nb);
  op_df_kernel<TX, TY, TZ><<<grid, 256, smem, ctx->stream>>>(static_cast<const double2 *>(X), sx,
                                                              static_cast<double2 *>(Y), sy, ctx->m0d.as<double>(),
                                                              ctx->kparam.as<KParam>(), act, ctx->logN);
  PC_CK_LAUNCH();
  return PC_OK;
}

// z-marching version (the blocking of opz_kernel in stencil.cu): a TX x TY column tile walks ZC planes with ring
// buffers of v (2 planes), e = M0 A' v (2 planes) and c = B v (2 planes).
template <int TX, int TY> constexpr size_t opz_df_smem_bytes() {
  return sizeof(cdf) * (size_t)(2 * 3 * (TY + 2) * (TX + 2) + 2 * 3 * (TY + 1) * (TX + 1) + 2 * (TY + 1) * (TX + 1));
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) opz_df_kernel(const double2 *__restrict__ X, long sx,
                                                         double2 *__restrict__ Y, long sy,
                                                         const double *__restrict__ m0,
                                                         const KParam *__restrict__ kp, const int *__restrict__ act,
                                                         int logN, int ZC) {
  constexpr int VX = TX + 2, VY = TY + 2, VP = VX * VY;
  constexpr int EX = TX + 1, EY = TY + 1, EP = EX * EY;
  constexpr int NT = TX * TY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cdf *vbuf = reinterpret_cast<cdf *>(smem_raw);
  cdf *ebuf = vbuf + 2 * 3 * VP;
  cdf *cbuf = ebuf + 2 * 3 * EP;
  const int N = 1 << logN, mask = N - 1;
  const long n = 1L << (3 * logN), plane = 1L << (2 * logN);
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int j = blockIdx.y;
  const int tilesX = N / TX, tilesY = N / TY;
  int t = blockIdx.x;
  const int x0 = (t % tilesX) * TX;
  t /= tilesX;
  const int y0 = (t % tilesY) * TY;
  const int zb = (t / tilesY) * ZC;
  const double2 *Xb = X + (long)b * sx + (long)j * 3 * n;
  double2 *Yb = Y + (long)b * sy + (long)j * 3 * n;
  const KParam &p = kp[b];
  const df kh0 = df_from(0.5 * p.k[0]), kh1 = df_from(0.5 * p.k[1]), kh2 = df_from(0.5 * p.k[2]);
  const df gam = df_from(p.gamma);
  const float ih = (float)N;
  const int tid = threadIdx.x;
  auto load_v = [&](int slot, int z) {
    const int gz = z & mask;
    cdf *vs = vbuf + slot * 3 * VP;
    for (int i = tid; i < 3 * VP; i += NT) {
      const int comp = i / VP, r = i - comp * VP, ly = r / VX, lx = r - ly * VX;
      const int gx = (x0 + lx - 1) & mask, gy = (y0 + ly - 1) & mask;
      vs[i] = cdf_from(Xb[comp * n + gz * plane + ((long)gy << logN) + gx]);
    }
  };
  auto make_e = [&](int eslot, int z, int sz, int szm) {
    const cdf *v0 = vbuf + sz * 3 * VP, *vm = vbuf + szm * 3 * VP;
    cdf *es = ebuf + eslot * 3 * EP;
    const int gz = z & mask;
    for (int i = tid; i < EP; i += NT) {
      const int ey = i / EX, ex = i - ey * EX;
      const int o = (ey + 1) * VX + ex + 1;
      const cdf v1 = v0[o], v2 = v0[VP + o], v3 = v0[2 * VP + o];
      const cdf d3v2 = dbwd_df(vm[VP + o], v2, ih, kh2);
      const cdf d2v3 = dbwd_df(v0[2 * VP + o - VX], v3, ih, kh1);
      const cdf d3v1 = dbwd_df(vm[o], v1, ih, kh2);
      const cdf d1v3 = dbwd_df(v0[2 * VP + o - 1], v3, ih, kh0);
      const cdf d2v1 = dbwd_df(v0[o - VX], v1, ih, kh1);
      const cdf d1v2 = dbwd_df(v0[VP + o - 1], v2, ih, kh0);
      const long gi = gz * plane + ((long)((y0 + ey) & mask) << logN) + ((x0 + ex) & mask);
      es[i] = cdf_scale(cdf_sub(d3v2, d2v3), df_from(m0[gi]));
      es[EP + i] = cdf_scale(cdf_sub(d1v3, d3v1), df_from(m0[n + gi]));
      es[2 * EP + i] = cdf_scale(cdf_sub(d2v1, d1v2), df_from(m0[2 * n + gi]));
    }
  };
  auto make_c = [&](int cslot, int sz, int szp) {
    const cdf *v0 = vbuf + sz * 3 * VP, *vp = vbuf + szp * 3 * VP;
    cdf *cs = cbuf + cslot * EP;
    for (int i = tid; i < EP; i += NT) {
      const int cy = i / EX, cx = i - cy * EX;
      const int o = cy * VX + cx;
      cdf cc = dfwd_df(v0[o], v0[o + 1], ih, kh0);
      cc = cdf_add(cc, dfwd_df(v0[VP + o], v0[VP + o + VX], ih, kh1));
      cc = cdf_add(cc, dfwd_df(v0[2 * VP + o], vp[2 * VP + o], ih, kh2));
      cs[i] = cc;
    }
  };
  load_v(0, zb - 1);
  load_v(1, zb);
  __syncthreads();
  make_e(0, zb, 1, 0);
  make_c(0, 0, 1);
  int sv = 1, se = 0, sc = 0;
  for (int z = zb; z < zb + ZC; ++z) {
    __syncthreads();
    load_v(1 - sv, z + 1);
    __syncthreads();
    make_e(1 - se, z + 1, 1 - sv, sv);
    make_c(1 - sc, sv, 1 - sv);
    __syncthreads();
    {
      const cdf *e0 = ebuf + se * 3 * EP, *e1p = ebuf + (1 - se) * 3 * EP;
      const cdf *cm = cbuf + sc * EP, *c0p = cbuf + (1 - sc) * EP;
      const int ly = tid / TX, lx = tid - ly * TX;
      const int eo = ly * EX + lx;
      const int co = (ly + 1) * EX + lx + 1;
      const cdf c0 = c0p[co];
      const cdf e1 = e0[eo], e2 = e0[EP + eo], e3 = e0[2 * EP + eo];
      cdf y1 = cdf_sub(dfwd_df(e3, e0[2 * EP + eo + EX], ih, kh1), dfwd_df(e2, e1p[EP + eo], ih, kh2));
      y1 = cdf_add(y1, cdf_scale(dbwd_df(c0p[co - 1], c0, ih, kh0), gam));
      cdf y2 = cdf_sub(dfwd_df(e1, e1p[eo], ih, kh2), dfwd_df(e3, e0[2 * EP + eo + 1], ih, kh0));
      y2 = cdf_add(y2, cdf_scale(dbwd_df(c0p[co - EX], c0, ih, kh1), gam));
      cdf y3 = cdf_sub(dfwd_df(e2, e0[EP + eo + 1], ih, kh0), dfwd_df(e1, e0[eo + EX], ih, kh1));
      y3 = cdf_add(y3, cdf_scale(dbwd_df(cm[co], c0, ih, kh2), gam));
      const long gi = (long)z * plane + ((long)(y0 + ly) << logN) + x0 + lx;
      Yb[gi] = cdf_to(y1);
      Yb[n + gi] = cdf_to(y2);
      Yb[2 * n + gi] = cdf_to(y3);
    }
    sv = 1 - sv;
    se = 1 - se;
    sc = 1 - sc;
  }
}

template <int TX, int TY>
static int launch_opz_df_t(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act) {
  constexpr size_t smem = opz_df_smem_bytes<TX, TY>();
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(opz_df_kernel<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  const int N = ctx->N;
  const long tiles = (long)(N / TX) * (N / TY) * m * nb;
  int ZC = N;
  while (ZC > 4 && tiles * (N / ZC) < 4L * 152 * 4) ZC >>= 1;
  dim3 grid((N / TX) * (N / TY) * (N / ZC), m, nb);
  opz_df_kernel<TX, TY><<<grid, TX * TY, smem, ctx->stream>>>(static_cast<const double2 *>(X), sx,
                                                               static_cast<double2 *>(Y), sy, ctx->m0d.as<double>(),
                                                               ctx->kparam.as<KParam>(), act, ctx->logN, ZC);
  PC_CK_LAUNCH();
  return PC_OK;
}

int launch_apply_op_df(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  const int N = ctx->N;
  if (N >= 32) return launch_opz_df_t<32, 8>(ctx, nb, m, X, sx, Y, sy, act);
  if (N == 16) return launch_op_df_t<16, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
  return launch_op_df_t<8, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
}

// ---------------------------------------------------------------- block update Y = X C + Z
constexpr int DF_QB = 8;

__global__ void __launch_bounds__(256) update_df_kernel(const double2 *__restrict__ X, long sx,
                                                       const double2 *__restrict__ Cm, long sc,
                                                       double2 *__restrict__ Y, long sy,
                                                       const float2 *__restrict__ Z, long sz, long L, int p, int q,
                                                       const int *__restrict__ act) {
  __shared__ cdf Cs[64][DF_QB];
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int j0 = blockIdx.y * DF_QB;
  const double2 *Cb = Cm + (long)b * sc;
  for (int i = threadIdx.x; i < p * DF_QB; i += blockDim.x) {
    const int r = i / DF_QB, c = i - r * DF_QB;
    Cs[r][c] = cdf_from((j0 + c < q) ? Cb[r * q + j0 + c] : make_double2(0.0, 0.0));
  }
  __syncthreads();
  const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const double2 *Xb = X + (long)b * sx;
  cdf acc[DF_QB];
#pragma unroll
  for (int c = 0; c < DF_QB; ++c) acc[c] = cdf{df{0.f, 0.f}, df{0.f, 0.f}};
  for (int i = 0; i < p; ++i) {
    const cdf xv = cdf_from(Xb[(long)i * L + l]);
#pragma unroll
    for (int c = 0; c < DF_QB; ++c) acc[c] = cdf_add(acc[c], cdf_mul(xv, Cs[i][c]));
  }
  double2 *Yb = Y + (long)b * sy;
  const float2 *Zb = Z ? Z + (long)b * sz : nullptr;
#pragma unroll
  for (int c = 0; c < DF_QB; ++c)
    if (j0 + c < q) {
      double2 v = cdf_to(acc[c]);
      if (Zb) {
        const float2 z = Zb[(long)(j0 + c) * L + l];
        v.x += (double)z.x;
        v.y += (double)z.y;
      }
      Yb[(long)(j0 + c) * L + l] = v;
    }
}

int launch_update_df(int nb, long L, int p, int q, const void *X, long sx, const void *C, long sc, void *Y, long sy,
                     const void *Z, long sz, cudaStream_t st, const int *act) {
  if (nb == 0 || q == 0) return PC_OK;
  dim3 grid((unsigned)((L + 255) / 256), (q + DF_QB - 1) / DF_QB, nb);
  update_df_kernel<<<grid, 256, 0, st>>>(static_cast<const double2 *>(X), sx, static_cast<const double2 *>(C), sc,
                                         static_cast<double2 *>(Y), sy, static_cast<const float2 *>(Z), sz, L, p, q,
                                         act);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ---------------------------------------------------------------- Gram pair G = X^H X, H = X^H AX
constexpr int DF_TL = 16;

template <int R>
__global__ void __launch_bounds__(1024) gram_df_kernel(const double2 *__restrict__ S, const double2 *__restrict__ AS,
                                                     long ss, long L, int p, long chunk,
                                                     double2 *__restrict__ partG, double2 *__restrict__ partH,
                                                     const int *__restrict__ act) {
  __shared__ cdf Ss[32][DF_TL + 1];
  __shared__ cdf As[32][DF_TL + 1];
  const int bi = blockIdx.z;
  const int b = act ? act[bi] : bi;
  const double2 *Sb = S + (long)b * ss;
  const double2 *Ab = AS + (long)b * ss;
  const int TD = blockDim.x;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TD + tx, nthr = TD * TD;
  const bool active = ty <= tx;
  cdf g[R][R], hh[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) g[r][c] = hh[r][c] = cdf{df{0.f, 0.f}, df{0.f, 0.f}};
  const long beg = (long)blockIdx.x * chunk, end = min(L, beg + chunk);
  for (long l0 = beg; l0 < end; l0 += DF_TL) {
    for (int i = tid; i < p * DF_TL; i += nthr) {
      const int col = i / DF_TL, t = i - col * DF_TL;
      const long l = l0 + t;
      double2 vs = make_double2(0.0, 0.0), va = vs;
      if (l < end) {
        vs = Sb[(long)col * L + l];
        va = Ab[(long)col * L + l];
      }
      Ss[col][t] = cdf_from(vs);
      As[col][t] = cdf_from(va);
    }
    __syncthreads();
    if (active) {
      for (int t = 0; t < DF_TL; ++t) {
        cdf a[R], bs[R], ba[R];
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
            g[r][c] = cdf_add(g[r][c], cdf_mulc(a[r], bs[c]));
            hh[r][c] = cdf_add(hh[r][c], cdf_mulc(a[r], ba[c]));
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
        partG[o + i * p + j] = cdf_to(g[r][c]);
        partH[o + i * p + j] = cdf_to(hh[r][c]);
      }
    }
}

// chunk sums of the upper triangle in FP64, mirrored (same layout as gram_pair_reduce_kernel)
__global__ void gram_df_reduce_kernel(const double2 *__restrict__ partG, const double2 *__restrict__ partH, int nchunk,
                                      int p, const int *__restrict__ act, double2 *__restrict__ G,
                                      double2 *__restrict__ H) {
  const int bi = blockIdx.x;
  const int b = act ? act[bi] : bi;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e - i * p;
    if (i > j) continue;
    double2 sg = make_double2(0.0, 0.0), sh = sg;
    for (int c = 0; c < nchunk; ++c) {
      sg = cadd(sg, partG[((long)bi * nchunk + c) * p * p + e]);
      sh = cadd(sh, partH[((long)bi * nchunk + c) * p * p + e]);
    }
    if (i == j) sg.y = sh.y = 0.0;
    G[(long)b * p * p + i * p + j] = sg;
    H[(long)b * p * p + i * p + j] = sh;
    G[(long)b * p * p + j * p + i] = make_double2(sg.x, -sg.y);
    H[(long)b * p * p + j * p + i] = make_double2(sh.x, -sh.y);
  }
}

static int df_chunks(int nb, long L) {
  long want = std::max<long>(1, (8L * 152 + nb - 1) / std::max(nb, 1));
  return (int)std::min<long>(std::min<long>(want, std::max<long>(1, L / 512)), 128);
}

size_t gram_df_scratch_bytes(int nb, long L, int p) {
  return 2 * sizeof(double2) * (size_t)nb * df_chunks(nb, L) * p * p;
}

int launch_gram_df(int nb, long L, int p, const void *S, const void *AS, long ss, void *G, void *H, void *scratch,
                   size_t scratch_bytes, cudaStream_t st, const int *act) {
  if (nb == 0 || p == 0) return PC_OK;
  if (p > 32 || gram_df_scratch_bytes(nb, L, p) > scratch_bytes) {
    set_error("gram_df: at most 32 columns and enough scratch");
    return PC_EINVAL;
  }
  const int nchunk = df_chunks(nb, L);
  long chunk = (L + nchunk - 1) / nchunk;
  chunk = (chunk + DF_TL - 1) / DF_TL * DF_TL;
  double2 *pG = static_cast<double2 *>(scratch), *pH = pG + (size_t)nb * nchunk * p * p;
  const double2 *Sd = static_cast<const double2 *>(S), *Ad = static_cast<const double2 *>(AS);
  // one output pair per thread (p x p threads, the upper triangle active): the double-float arithmetic is the
  // bottleneck, so parallelism matters more than register reuse
  gram_df_kernel<1><<<dim3(nchunk, 1, nb), dim3(p, p), 0, st>>>(Sd, Ad, ss, L, p, chunk, pG, pH, act);
  PC_CK_LAUNCH();
  gram_df_reduce_kernel<<<nb, 256, 0, st>>>(pG, pH, nchunk, p, act, static_cast<double2 *>(G),
                                            static_cast<double2 *>(H));
  PC_CK_LAUNCH();
  return PC_OK;
}

}  // namespace pc
