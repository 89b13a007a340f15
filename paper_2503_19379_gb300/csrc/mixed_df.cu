// The FP64-accurate kernels of the mixed-precision solve, in double-float arithmetic (dfloat.cuh) on the FP32 pipe
// (GB300: 75 TFLOP/s FP32 against 1.2 TFLOP/s FP64). The solver's block X is stored as double-float pairs (PC_DFS,
// one float4 per complex element), so these kernels do no FP64 arithmetic at all; the public stencil entry point
// takes complex128 and converts on load and store.
//   op_df_kernel / opz_df_kernel  AX = Op X (the stencil of stencil.cu; differences, shifts, M0, gamma in
//                     double-float), or, in the solver, the residual epilogue: R = AX - X Theta and complex64 copies
//                     of R, X and AX, plus column norms (AX itself is not stored)
//   update_df_kernel  X' = X C + Z  (Z: the complex64 correction [W P] coef_{W,P})
//   gram_df_kernel    G = X^H X  (upper triangle, Hermitian mirror)
#include <cmath>
#include <type_traits>

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

// Residual epilogue of the stencil (the mixed solve's phase 2): instead of AX the kernel writes, per point,
// r = AX - theta_j X rounded to complex64 (twice: the preconditioner's input slot and the persistent copy used by
// the Rayleigh-Ritz coupling), complex64 copies of X and AX for the complex64 Gram products, and per-block partial
// sums of |r|^2 and |x|^2 (FP32 per thread, FP64 per block), reduced per column by residual_reduce.
struct ResidArgs {
  const double *theta;  // [nb][m]
  int m;
  float2 *R1, *R2, *X32, *AX32;
  long sr1, sr2, sx32, sax32;
  double *part;  // [nb][m][blocks per field][2]
};

__device__ __forceinline__ float2 cdf_round(cdf a) { return make_float2(a.re.hi + a.re.lo, a.im.hi + a.im.lo); }
__device__ __forceinline__ df ld_m0(const float2 *p) {
  const float2 v = *p;
  return df{v.x, v.y};
}

// writes the three components of one point; returns |r|^2 and |x|^2 contributions
__device__ __forceinline__ void resid_point(const ResidArgs &ra, int b, int j, long n, long gi, df th, const cdf (&y)[3],
                                            const cdf (&x)[3], float &sr, float &sxx) {
  const long L = 3 * n;
  float2 *r1 = ra.R1 + (long)b * ra.sr1 + (long)j * L, *r2 = ra.R2 + (long)b * ra.sr2 + (long)j * L;
  float2 *x32 = ra.X32 + (long)b * ra.sx32 + (long)j * L, *ax32 = ra.AX32 + (long)b * ra.sax32 + (long)j * L;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cdf r = cdf_sub(y[c], cdf_scale(x[c], th));
    const float2 rf = cdf_round(r), xf = make_float2(x[c].re.hi, x[c].im.hi);
    const long o = c * n + gi;
    r1[o] = rf;
    r2[o] = rf;
    x32[o] = xf;
    ax32[o] = cdf_round(y[c]);
    sr += rf.x * rf.x + rf.y * rf.y;
    sxx += xf.x * xf.x + xf.y * xf.y;
  }
}

// block sum of (sr, sxx) into the partial-sum slot of this block
__device__ __forceinline__ void resid_block_sum(const ResidArgs &ra, float sr, float sxx) {
  __shared__ double red[2][32];
  double a = sr, c = sxx;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = a;
    red[1][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int i = 0; i < nw; ++i) {
      s0 += red[0][i];
      s1 += red[1][i];
    }
    double *o = ra.part + (((long)blockIdx.z * ra.m + blockIdx.y) * gridDim.x + blockIdx.x) * 2;
    o[0] = s0;
    o[1] = s1;
  }
}

template <int TX, int TY, int TZ> constexpr size_t op_df_smem_bytes() {
  return sizeof(cdf) * (size_t)(3 * (TZ + 2) * (TY + 2) * (TX + 2) + 3 * (TZ + 1) * (TY + 1) * (TX + 1) +
                                (TZ + 1) * (TY + 1) * (TX + 1));
}

// Same tiling as op_kernel (stencil.cu): a face tile with a one-point halo, e = M0 A' v on the tile grown upward,
// c = B v on the tile grown downward, then y = A e + gamma B' c. The grid spacing factor ih = N is a power of two,
// so scaling by it is exact in double-float.
// The block is complex128 (converted on load and store) for the public entry point, double-float pairs (PC_DFS) for
// the solver's fused residual version.
template <bool RES> using df_store_t = typename std::conditional<RES, float4, double2>::type;

__device__ __forceinline__ df kp_df(float hi, float lo) { return df{hi, lo}; }

template <int TX, int TY, int TZ, bool RES>
__global__ void __launch_bounds__(256) op_df_kernel(const df_store_t<RES> *__restrict__ X, long sx,
                                                    df_store_t<RES> *__restrict__ Y, long sy,
                                                    const float2 *__restrict__ m0, const KParam *__restrict__ kp,
                                                    const int *__restrict__ act, int logN, const ResidArgs ra) {
  using XS = df_store_t<RES>;
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
  const XS *Xb = X + (long)b * sx + (long)j * 3 * n;
  XS *Yb = Y + (long)b * sy + (long)j * 3 * n;
  const KParam p = kp[b];
  const df kh0 = kp_df(p.khf[0], p.khl[0]), kh1 = kp_df(p.khf[1], p.khl[1]), kh2 = kp_df(p.khf[2], p.khl[2]);
  const df gam = kp_df(p.gammaf, p.gammal);
  const float ih = (float)N;

  for (int i = threadIdx.x; i < 3 * VZ * VY * VX; i += blockDim.x) {
    int lx = i % VX, r = i / VX;
    int ly = r % VY;
    r /= VY;
    int lz = r % VZ, comp = r / VZ;
    int gx = (x0 + lx - 1) & mask, gy = (y0 + ly - 1) & mask, gz = (z0 + lz - 1) & mask;
    v[i] = ld_cdf(Xb + comp * n + ((long)gz << (2 * logN)) + ((long)gy << logN) + gx);
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
    e[eo] = cdf_scale(cdf_sub(d3v2, d2v3), ld_m0(m0 + gi));
    e[EZ * EY * EX + eo] = cdf_scale(cdf_sub(d1v3, d3v1), ld_m0(m0 + n + gi));
    e[2 * EZ * EY * EX + eo] = cdf_scale(cdf_sub(d2v1, d1v2), ld_m0(m0 + 2 * n + gi));
#define WW(comp, dz, dy, dx) v[(((comp) * VZ + ez + (dz)) * VY + ey + (dy)) * VX + ex + (dx)]
    cdf cc = dfwd_df(WW(0, 0, 0, 0), WW(0, 0, 0, 1), ih, kh0);
    cc = cdf_add(cc, dfwd_df(WW(1, 0, 0, 0), WW(1, 0, 1, 0), ih, kh1));
    cc = cdf_add(cc, dfwd_df(WW(2, 0, 0, 0), WW(2, 1, 0, 0), ih, kh2));
#undef WW
    c[eo] = cc;
  }
  __syncthreads();
  float sr = 0.f, sxx = 0.f;
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
    if constexpr (RES) {
#define XV(comp) v[(((comp) * VZ + lz + 1) * VY + ly + 1) * VX + lx + 1]
      const cdf yv[3] = {y1, y2, y3}, xv[3] = {XV(0), XV(1), XV(2)};
#undef XV
      resid_point(ra, b, j, n, gi, df_from(ra.theta[(long)b * ra.m + j]), yv, xv, sr, sxx);
    } else {
      st_cdf(Yb + gi, y1);
      st_cdf(Yb + n + gi, y2);
      st_cdf(Yb + 2 * n + gi, y3);
    }
  }
  if constexpr (RES) resid_block_sum(ra, sr, sxx);
}

template <int TX, int TY, int TZ, bool RES>
static int launch_op_df_t(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act,
                          const ResidArgs &ra, int *nchunk) {
  constexpr size_t smem = op_df_smem_bytes<TX, TY, TZ>();
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(op_df_kernel<TX, TY, TZ, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
    configured = true;
  }
  const int N = ctx->N;
  dim3 grid((N / TX) * (N / TY) * (N / TZ), m, nb);
  *nchunk = (int)grid.x;
  if (RES && ra.part == nullptr) return PC_OK;  // sizing call
  op_df_kernel<TX, TY, TZ, RES><<<grid, 256, smem, ctx->stream>>>(
      static_cast<const df_store_t<RES> *>(X), sx, static_cast<df_store_t<RES> *>(Y), sy, ctx->m0p.as<float2>(),
      ctx->kparam.as<KParam>(), act, ctx->logN, ra);
  PC_CK_LAUNCH();
  return PC_OK;
}

// z-marching version (the blocking of opz_kernel in stencil.cu): a TX x TY column tile walks ZC planes with ring
// buffers of v (2 planes), e = M0 A' v (2 planes) and c = B v (2 planes).
template <int TX, int TY> constexpr size_t opz_df_smem_bytes() {
  return sizeof(cdf) * (size_t)(2 * 3 * (TY + 2) * (TX + 2) + 2 * 3 * (TY + 1) * (TX + 1) + 2 * (TY + 1) * (TX + 1));
}

template <int TX, int TY, bool RES>
__global__ void __launch_bounds__(TX * TY) opz_df_kernel(const df_store_t<RES> *__restrict__ X, long sx,
                                                         df_store_t<RES> *__restrict__ Y, long sy,
                                                         const float2 *__restrict__ m0,
                                                         const KParam *__restrict__ kp, const int *__restrict__ act,
                                                         int logN, int ZC, const ResidArgs ra) {
  using XS = df_store_t<RES>;
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
  const XS *Xb = X + (long)b * sx + (long)j * 3 * n;
  XS *Yb = Y + (long)b * sy + (long)j * 3 * n;
  const KParam &p = kp[b];
  const df kh0 = kp_df(p.khf[0], p.khl[0]), kh1 = kp_df(p.khf[1], p.khl[1]), kh2 = kp_df(p.khf[2], p.khl[2]);
  const df gam = kp_df(p.gammaf, p.gammal);
  const float ih = (float)N;
  const int tid = threadIdx.x;
  auto load_v = [&](int slot, int z) {
    const int gz = z & mask;
    cdf *vs = vbuf + slot * 3 * VP;
    for (int i = tid; i < 3 * VP; i += NT) {
      const int comp = i / VP, r = i - comp * VP, ly = r / VX, lx = r - ly * VX;
      const int gx = (x0 + lx - 1) & mask, gy = (y0 + ly - 1) & mask;
      vs[i] = ld_cdf(Xb + comp * n + gz * plane + ((long)gy << logN) + gx);
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
      es[i] = cdf_scale(cdf_sub(d3v2, d2v3), ld_m0(m0 + gi));
      es[EP + i] = cdf_scale(cdf_sub(d1v3, d3v1), ld_m0(m0 + n + gi));
      es[2 * EP + i] = cdf_scale(cdf_sub(d2v1, d1v2), ld_m0(m0 + 2 * n + gi));
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
  float sr = 0.f, sxx = 0.f;
  const df th = RES ? df_from(ra.theta[(long)b * ra.m + j]) : df{0.f, 0.f};
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
      if constexpr (RES) {
        const cdf *v0 = vbuf + sv * 3 * VP;  // plane z
        const int o = (ly + 1) * VX + lx + 1;
        const cdf yv[3] = {y1, y2, y3}, xv[3] = {v0[o], v0[VP + o], v0[2 * VP + o]};
        resid_point(ra, b, j, n, gi, th, yv, xv, sr, sxx);
      } else {
        st_cdf(Yb + gi, y1);
        st_cdf(Yb + n + gi, y2);
        st_cdf(Yb + 2 * n + gi, y3);
      }
    }
    sv = 1 - sv;
    se = 1 - se;
    sc = 1 - sc;
  }
  if constexpr (RES) resid_block_sum(ra, sr, sxx);
}

template <int TX, int TY, bool RES>
static int launch_opz_df_t(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act,
                           const ResidArgs &ra, int *nchunk) {
  constexpr size_t smem = opz_df_smem_bytes<TX, TY>();
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(opz_df_kernel<TX, TY, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  const int N = ctx->N;
  const long tiles = (long)(N / TX) * (N / TY) * m * nb;
  int ZC = N;
  while (ZC > 4 && tiles * (N / ZC) < 16L * sm_count()) ZC >>= 1;
  dim3 grid((N / TX) * (N / TY) * (N / ZC), m, nb);
  *nchunk = (int)grid.x;
  if (RES && ra.part == nullptr) return PC_OK;  // sizing call
  opz_df_kernel<TX, TY, RES><<<grid, TX * TY, smem, ctx->stream>>>(
      static_cast<const df_store_t<RES> *>(X), sx, static_cast<df_store_t<RES> *>(Y), sy, ctx->m0p.as<float2>(),
      ctx->kparam.as<KParam>(), act, ctx->logN, ZC, ra);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ---------------------------------------------------------------- general lattice (Section 4.2.2)
// D_hat_a f = sum_j (b_ja / h)(f_{r+e_j} - f_r) + i kh_a (f_r + f_{r+e_a}) and its adjoint
// D_hat_a' g = sum_j (b_ja / h)(g_{r-e_j} - g_r) - i kh_a (g_{r-e_a} + g_r), second order, in double-float; the
// weights b_ja / h are double-float pairs. Two passes through a per-stream scratch block (e = M0 A' v, c = B v as
// double-float pairs, then y = A e + gamma B' c), the second with the residual epilogue of the cubic kernels.
struct LatDF {
  df bh[9];  // bh[3 j + a] = b_ja N
};

__device__ __forceinline__ long lat_nb(long i, int axis, int off, int logN) {
  const int N = 1 << logN, mask = N - 1;
  int x = (int)(i & mask), y = (int)((i >> logN) & mask), z = (int)(i >> (2 * logN));
  if (axis == 0) x = (x + off) & mask;
  else if (axis == 1) y = (y + off) & mask;
  else z = (z + off) & mask;
  return ((long)z << (2 * logN)) + ((long)y << logN) + x;
}

// D_hat_a (adj = false) or D_hat_a' (adj = true) of field f at point i; f[...] read through ld_cdf
template <typename S>
__device__ __forceinline__ cdf dlat_df(const S *__restrict__ f, long i, int a, bool adj, int logN, const LatDF &lt,
                                       df kh) {
  const cdf f0 = ld_cdf(f + i);
  cdf acc = cdf{df{0.f, 0.f}, df{0.f, 0.f}}, sm = acc;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const cdf fj = ld_cdf(f + lat_nb(i, j, adj ? -1 : 1, logN));
    acc = cdf_add(acc, cdf_scale(cdf_sub(fj, f0), lt.bh[3 * j + a]));
    if (j == a) sm = cdf_add(fj, f0);
  }
  // acc + i kh sm (forward) or acc - i kh sm (adjoint)
  const df sr = df_mul(kh, sm.re), si = df_mul(kh, sm.im);
  return adj ? cdf{df_add(acc.re, si), df_sub(acc.im, sr)} : cdf{df_sub(acc.re, si), df_add(acc.im, sr)};
}

// pass 1: E (3 fields) and Cc (1 field) of column j of k-point act[bz], double-float pairs. grid (n / 256, m, nb)
template <typename XS>
__global__ void __launch_bounds__(256) lat_df_half_kernel(const XS *__restrict__ X, long sx, float4 *__restrict__ E,
                                                          const float2 *__restrict__ m0, const KParam *__restrict__ kp,
                                                          const int *__restrict__ act, int logN, const LatDF lt) {
  const long n = 1L << (3 * logN);
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int bz = blockIdx.z, j = blockIdx.y, m = gridDim.y;
  const int b = act ? act[bz] : bz;
  const KParam &p = kp[b];
  const df kh0 = kp_df(p.khf[0], p.khl[0]), kh1 = kp_df(p.khf[1], p.khl[1]), kh2 = kp_df(p.khf[2], p.khl[2]);
  const XS *v1 = X + (long)b * sx + (long)j * 3 * n, *v2 = v1 + n, *v3 = v2 + n;
  const cdf e1 = cdf_scale(cdf_sub(dlat_df(v2, i, 2, true, logN, lt, kh2), dlat_df(v3, i, 1, true, logN, lt, kh1)),
                           ld_m0(m0 + i));
  const cdf e2 = cdf_scale(cdf_sub(dlat_df(v3, i, 0, true, logN, lt, kh0), dlat_df(v1, i, 2, true, logN, lt, kh2)),
                           ld_m0(m0 + n + i));
  const cdf e3 = cdf_scale(cdf_sub(dlat_df(v1, i, 1, true, logN, lt, kh1), dlat_df(v2, i, 0, true, logN, lt, kh0)),
                           ld_m0(m0 + 2 * n + i));
  const cdf c = cdf_add(cdf_add(dlat_df(v1, i, 0, false, logN, lt, kh0), dlat_df(v2, i, 1, false, logN, lt, kh1)),
                        dlat_df(v3, i, 2, false, logN, lt, kh2));
  float4 *eb = E + ((long)bz * m + j) * 4 * n;
  st_cdf(eb + i, e1);
  st_cdf(eb + n + i, e2);
  st_cdf(eb + 2 * n + i, e3);
  st_cdf(eb + 3 * n + i, c);
}

// pass 2: y = A e + gamma B' c, stored (RES = false) or reduced to the residual epilogue (RES = true; every thread
// of the block takes part in its block sum). grid (n / 256, m, nb), 256 threads
template <bool RES>
__global__ void __launch_bounds__(256) lat_df_full_kernel(const float4 *__restrict__ E, const df_store_t<RES> *__restrict__ X,
                                                          long sx, df_store_t<RES> *__restrict__ Y, long sy,
                                                          const KParam *__restrict__ kp, const int *__restrict__ act,
                                                          int logN, const LatDF lt, const ResidArgs ra) {
  const long n = 1L << (3 * logN);
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int bz = blockIdx.z, j = blockIdx.y, m = gridDim.y;
  const int b = act ? act[bz] : bz;
  const KParam &p = kp[b];
  float sr = 0.f, sxx = 0.f;
  if (i < n) {
    const df kh0 = kp_df(p.khf[0], p.khl[0]), kh1 = kp_df(p.khf[1], p.khl[1]), kh2 = kp_df(p.khf[2], p.khl[2]);
    const df gam = kp_df(p.gammaf, p.gammal);
    const float4 *e1 = E + ((long)bz * m + j) * 4 * n, *e2 = e1 + n, *e3 = e2 + n, *c = e3 + n;
    cdf y1 = cdf_sub(dlat_df(e3, i, 1, false, logN, lt, kh1), dlat_df(e2, i, 2, false, logN, lt, kh2));
    y1 = cdf_add(y1, cdf_scale(dlat_df(c, i, 0, true, logN, lt, kh0), gam));
    cdf y2 = cdf_sub(dlat_df(e1, i, 2, false, logN, lt, kh2), dlat_df(e3, i, 0, false, logN, lt, kh0));
    y2 = cdf_add(y2, cdf_scale(dlat_df(c, i, 1, true, logN, lt, kh1), gam));
    cdf y3 = cdf_sub(dlat_df(e2, i, 0, false, logN, lt, kh0), dlat_df(e1, i, 1, false, logN, lt, kh1));
    y3 = cdf_add(y3, cdf_scale(dlat_df(c, i, 2, true, logN, lt, kh2), gam));
    if constexpr (RES) {
      const df_store_t<RES> *xb = X + (long)b * sx + (long)j * 3 * n;
      const cdf yv[3] = {y1, y2, y3}, xv[3] = {ld_cdf(xb + i), ld_cdf(xb + n + i), ld_cdf(xb + 2 * n + i)};
      const df th = df_from(ra.theta[(long)b * ra.m + j]);
      resid_point(ra, b, j, n, i, th, yv, xv, sr, sxx);
    } else {
      df_store_t<RES> *yb = Y + (long)b * sy + (long)j * 3 * n;
      st_cdf(yb + i, y1);
      st_cdf(yb + n + i, y2);
      st_cdf(yb + 2 * n + i, y3);
    }
  }
  if constexpr (RES) resid_block_sum(ra, sr, sxx);
}

template <bool RES>
int launch_op_df_lat(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act,
                     const ResidArgs &ra, int *nchunk) {
  const long n = ctx->n;
  const dim3 grid((unsigned)((n + 255) / 256), m, nb);
  *nchunk = (int)grid.x;
  if (RES && ra.part == nullptr) return PC_OK;  // sizing call
  LatDF lt;
  for (int q = 0; q < 9; ++q) {
    const double v = ctx->binv[q] * (double)ctx->N;
    lt.bh[q].hi = (float)v;
    lt.bh[q].lo = (float)(v - (double)lt.bh[q].hi);
  }
  DevBuf &ks = kscratch_for(ctx);
  PC_CK(ks.reserve(sizeof(float4) * 4 * (size_t)n * m * nb));
  float4 *E = ks.as<float4>();
  using XS = df_store_t<RES>;
  lat_df_half_kernel<XS><<<grid, 256, 0, ctx->stream>>>(static_cast<const XS *>(X), sx, E, ctx->m0p.as<float2>(),
                                                         ctx->kparam.as<KParam>(), act, ctx->logN, lt);
  PC_CK_LAUNCH();
  lat_df_full_kernel<RES><<<grid, 256, 0, ctx->stream>>>(E, static_cast<const XS *>(X), sx, static_cast<XS *>(Y), sy,
                                                          ctx->kparam.as<KParam>(), act, ctx->logN, lt, ra);
  PC_CK_LAUNCH();
  return PC_OK;
}

template <bool RES>
static int op_df_dispatch(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act,
                          const ResidArgs &ra, int *nchunk) {
  if (ctx->lat) return launch_op_df_lat<RES>(ctx, nb, m, X, sx, Y, sy, act, ra, nchunk);
  const int N = ctx->N;
  if (N >= 32) return launch_opz_df_t<32, 8, RES>(ctx, nb, m, X, sx, Y, sy, act, ra, nchunk);
  if (N == 16) return launch_op_df_t<16, 4, 4, RES>(ctx, nb, m, X, sx, Y, sy, act, ra, nchunk);
  return launch_op_df_t<8, 4, 4, RES>(ctx, nb, m, X, sx, Y, sy, act, ra, nchunk);
}

int launch_apply_op_df(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  if (ctx->opts.order != 1) {
    set_error("double-float stencil: second order (order 1) only");
    return PC_EUNSUPPORTED;
  }
  int nchunk = 0;
  return op_df_dispatch<false>(ctx, nb, m, X, sx, Y, sy, act, ResidArgs{}, &nchunk);
}

size_t op_df_resid_scratch_bytes(pc_ctx *ctx, int nb, int m) {
  int nchunk = 0;
  op_df_dispatch<true>(ctx, nb, m, nullptr, 0, nullptr, 0, nullptr, ResidArgs{}, &nchunk);
  return sizeof(double) * 2 * (size_t)nb * m * nchunk;
}

int launch_op_df_resid(pc_ctx *ctx, int nb, int m, const void *X, long sx, const double *theta, void *R1, long sr1,
                       void *R2, long sr2, void *X32, long sx32, void *AX32, long sax32, double *norms, void *scratch,
                       size_t scratch_bytes, const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  if (op_df_resid_scratch_bytes(ctx, nb, m) > scratch_bytes) {
    set_error("op_df_resid: scratch too small");
    return PC_EINVAL;
  }
  ResidArgs ra{theta, m, static_cast<float2 *>(R1), static_cast<float2 *>(R2), static_cast<float2 *>(X32),
               static_cast<float2 *>(AX32), sr1, sr2, sx32, sax32, static_cast<double *>(scratch)};
  int nchunk = 0;
  int rc = op_df_dispatch<true>(ctx, nb, m, X, sx, nullptr, 0, act, ra, &nchunk);
  if (rc) return rc;
  launch_residual_reduce(nb, nchunk, m, static_cast<const double *>(scratch), act, norms, ctx->stream);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ---------------------------------------------------------------- block update Y = X C + Z
// One row per thread, QB output columns per block row of the grid (QB from the column count so that few columns
// are computed for nothing: 19 columns take two blocks of 10, not three of 8). Coefficients in shared memory as
// double-float (re, im, -im); each term is a dfsum multiply-add (12 FP32 operations per real term).
template <int QB>
__global__ void __launch_bounds__(256) update_df_kernel(const float4 *__restrict__ X, long sx,
                                                       const double2 *__restrict__ Cm, long sc,
                                                       float4 *__restrict__ Y, long sy,
                                                       const float2 *__restrict__ Z, long sz, long L, int p, int q,
                                                       const int *__restrict__ act) {
  __shared__ df Cs[64][QB][3];  // (re, im, -im) of C[i][j0 + c]
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int j0 = blockIdx.y * QB;
  const double2 *Cb = Cm + (long)b * sc;
  for (int i = threadIdx.x; i < p * QB; i += blockDim.x) {
    const int r = i / QB, c = i - r * QB;
    const double2 v = (j0 + c < q) ? Cb[r * q + j0 + c] : make_double2(0.0, 0.0);
    Cs[r][c][0] = df_from(v.x);
    Cs[r][c][1] = df_from(v.y);
    Cs[r][c][2] = df_from(-v.y);
  }
  __syncthreads();
  const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const float4 *Xb = X + (long)b * sx;
  dfsum re[QB], im[QB];
#pragma unroll
  for (int c = 0; c < QB; ++c) re[c] = im[c] = dfsum{0.f, 0.f};
  for (int i = 0; i < p; ++i) {
    const cdf xv = ld_cdf(Xb + (long)i * L + l);
#pragma unroll
    for (int c = 0; c < QB; ++c) {
      // (xr + i xi)(cr + i ci) = (xr cr - xi ci) + i (xr ci + xi cr)
      dfsum_mac(re[c], xv.re, Cs[i][c][0]);
      dfsum_mac(re[c], xv.im, Cs[i][c][2]);
      dfsum_mac(im[c], xv.re, Cs[i][c][1]);
      dfsum_mac(im[c], xv.im, Cs[i][c][0]);
    }
  }
  float4 *Yb = Y + (long)b * sy;
  const float2 *Zb = Z ? Z + (long)b * sz : nullptr;
#pragma unroll
  for (int c = 0; c < QB; ++c)
    if (j0 + c < q) {
      if (Zb) {
        const float2 z = Zb[(long)(j0 + c) * L + l];
        dfsum_addf(re[c], z.x);
        dfsum_addf(im[c], z.y);
      }
      st_cdf(Yb + (long)(j0 + c) * L + l, cdf{dfsum_value(re[c]), dfsum_value(im[c])});
    }
}

int launch_update_df(int nb, long L, int p, int q, const void *X, long sx, const void *C, long sc, void *Y, long sy,
                     const void *Z, long sz, cudaStream_t st, const int *act) {
  if (nb == 0 || q == 0) return PC_OK;
  if (p > 64) {
    set_error("update_df: at most 64 input columns");
    return PC_EINVAL;
  }
  // blocks of columns: 8 wide unless 10 wastes fewer (q = 19: 2 x 10 instead of 3 x 8)
  const int nb8 = (q + 7) / 8, nb10 = (q + 9) / 10;
  const bool wide = nb10 * 10 < nb8 * 8;
  const unsigned gx = (unsigned)((L + 255) / 256);
  if (wide)
    update_df_kernel<10><<<dim3(gx, nb10, nb), 256, 0, st>>>(static_cast<const float4 *>(X), sx,
                                                             static_cast<const double2 *>(C), sc, static_cast<float4 *>(Y),
                                                             sy, static_cast<const float2 *>(Z), sz, L, p, q, act);
  else
    update_df_kernel<8><<<dim3(gx, nb8, nb), 256, 0, st>>>(static_cast<const float4 *>(X), sx,
                                                           static_cast<const double2 *>(C), sc, static_cast<float4 *>(Y),
                                                           sy, static_cast<const float2 *>(Z), sz, L, p, q, act);
  PC_CK_LAUNCH();
  return PC_OK;
}

// ---------------------------------------------------------------- Gram G = X^H X of the FP64 block
// (X^H AX is not formed here: the mixed solve takes it as Theta X^H X + R^H X, R = AX - X Theta.)
constexpr int DF_TL = 32;

// One thread per upper-triangle entry (i <= j): p(p+1)/2 threads; grid (nchunk, 1, nb).
__global__ void __launch_bounds__(528) gram_df_kernel(const float4 *__restrict__ X, long sx, long L, int p,
                                                     long chunk, double2 *__restrict__ part,
                                                     const int *__restrict__ act) {
  __shared__ cdf Xs[32][DF_TL + 1];
  __shared__ unsigned char pi[528], pj[528];
  const int bi = blockIdx.z;
  const int b = act ? act[bi] : bi;
  const float4 *Xb = X + (long)b * sx;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    int t = 0;
    for (int i = 0; i < p; ++i)
      for (int j = i; j < p; ++j, ++t) {
        pi[t] = (unsigned char)i;
        pj[t] = (unsigned char)j;
      }
  }
  __syncthreads();
  const int i = pi[tid], j = pj[tid];
  // two independent sums (even and odd rows of each tile): twice the instruction-level parallelism of one chain
  dfsum re0{0.f, 0.f}, im0{0.f, 0.f}, re1{0.f, 0.f}, im1{0.f, 0.f};
  const long beg = (long)blockIdx.x * chunk, end = min(L, beg + chunk);
  for (long l0 = beg; l0 < end; l0 += DF_TL) {
    for (int e = tid; e < p * DF_TL; e += nthr) {
      const int col = e / DF_TL, t = e - col * DF_TL;
      const long l = l0 + t;
      Xs[col][t] = l < end ? ld_cdf(Xb + (long)col * L + l) : cdf{df{0.f, 0.f}, df{0.f, 0.f}};
    }
    __syncthreads();
#pragma unroll 2
    for (int t = 0; t < DF_TL; t += 2) {
      const cdf a = Xs[i][t], c = Xs[j][t], a1 = Xs[i][t + 1], c1 = Xs[j][t + 1];
      // conj(a) c = (ar cr + ai ci) + i (ar ci - ai cr)
      dfsum_mac(re0, a.re, c.re);
      dfsum_mac(re1, a1.re, c1.re);
      dfsum_mac(im0, a.re, c.im);
      dfsum_mac(im1, a1.re, c1.im);
      dfsum_mac(re0, a.im, c.im);
      dfsum_mac(re1, a1.im, c1.im);
      dfsum_mac(im0, df_neg(a.im), c.re);
      dfsum_mac(im1, df_neg(a1.im), c1.re);
    }
    __syncthreads();
  }
  const df re = df_add(dfsum_value(re0), dfsum_value(re1)), im = df_add(dfsum_value(im0), dfsum_value(im1));
  part[((long)bi * gridDim.x + blockIdx.x) * p * p + i * p + j] = make_double2(df_to(re), df_to(im));
}

// chunk sums of the upper triangle in FP64, mirrored
__global__ void gram_df_reduce_kernel(const double2 *__restrict__ part, int nchunk, int p, const int *__restrict__ act,
                                      double2 *__restrict__ G) {
  const int bi = blockIdx.x;
  const int b = act ? act[bi] : bi;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e - i * p;
    if (i > j) continue;
    double2 sg = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunk; ++c) sg = cadd(sg, part[((long)bi * nchunk + c) * p * p + e]);
    if (i == j) sg.y = 0.0;
    G[(long)b * p * p + i * p + j] = sg;
    G[(long)b * p * p + j * p + i] = make_double2(sg.x, -sg.y);
  }
}

static int df_chunks(int nb, long L) {
  long want = std::max<long>(1, (8L * sm_count() + nb - 1) / std::max(nb, 1));
  return (int)std::min<long>(std::min<long>(want, std::max<long>(1, L / 512)), 128);
}

size_t gram_df_scratch_bytes(int nb, long L, int p) {
  return sizeof(double2) * (size_t)nb * df_chunks(nb, L) * p * p;
}

int launch_gram_df(int nb, long L, int p, const void *X, long sx, void *G, void *scratch, size_t scratch_bytes,
                   cudaStream_t st, const int *act) {
  if (nb == 0 || p == 0) return PC_OK;
  if (p > 32 || gram_df_scratch_bytes(nb, L, p) > scratch_bytes) {
    set_error("gram_df: at most 32 columns and enough scratch");
    return PC_EINVAL;
  }
  const int nchunk = df_chunks(nb, L);
  long chunk = (L + nchunk - 1) / nchunk;
  chunk = (chunk + DF_TL - 1) / DF_TL * DF_TL;
  double2 *part = static_cast<double2 *>(scratch);
  gram_df_kernel<<<dim3(nchunk, 1, nb), p * (p + 1) / 2, 0, st>>>(static_cast<const float4 *>(X), sx, L, p, chunk,
                                                                   part, act);
  PC_CK_LAUNCH();
  gram_df_reduce_kernel<<<nb, 256, 0, st>>>(part, nchunk, p, act, static_cast<double2 *>(G));
  PC_CK_LAUNCH();
  return PC_OK;
}

}  // namespace pc
