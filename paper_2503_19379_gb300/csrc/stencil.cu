// Matrix-free compensated operator Op = A M0 A' + gamma B'B (eq. Ker_comp) on the staggered MFD grid, second-order
// stencils (Section 4.1.2, eqs. stencils, blocks, discrete_2nd_block, derived_uniform_grid), and the half applies
// A' x, B x used by Algorithm 4.1.
//
// Along axis i the shifted differences are, with kh = k_i / 2 and ih = 1/h,
//   (D_i f)_r  = ih (f_{r+1} - f_r) + i kh (f_r + f_{r+1})          faces -> cells, edges -> faces (forward)
//   (D_i' g)_r = ih (g_{r-1} - g_r) - i kh (g_{r-1} + g_r)          the conjugate transpose (backward)
// A = [[0,-D3,D2],[D3,0,-D1],[-D2,D1,0]], A' = [[0,D3',-D2'],[-D3',0,D1'],[D2',-D1',0]], B = [D1 D2 D3],
// B' = [D1'; D2'; D3'].
//
// The fused kernel stages a face tile with a one-point halo in shared memory, forms e = M0 A' v on the tile grown by
// one point upward and c = B v on the tile grown by one point downward, then writes y = A e + gamma B' c. Every
// input face value is read from global memory once per tile (plus halo).
#include <cstdio>

#include "dfloat.cuh"
#include "pc_internal.cuh"

namespace pc {

template <typename C, typename T> __device__ __forceinline__ C dfwd(C f0, C f1, T ih, T kh) {
  T ar = f1.x - f0.x, ai = f1.y - f0.y;
  T sr = f0.x + f1.x, si = f0.y + f1.y;
  return cmake<C>(ih * ar - kh * si, ih * ai + kh * sr);
}
template <typename C, typename T> __device__ __forceinline__ C dbwd(C gm, C g0, T ih, T kh) {
  T ar = gm.x - g0.x, ai = gm.y - g0.y;
  T sr = gm.x + g0.x, si = gm.y + g0.y;
  return cmake<C>(ih * ar + kh * si, ih * ai - kh * sr);
}

template <typename T, int TX, int TY, int TZ> constexpr size_t op_smem_bytes() {
  return sizeof(cplx<T>) * (size_t)(3 * (TZ + 2) * (TY + 2) * (TX + 2) + 3 * (TZ + 1) * (TY + 1) * (TX + 1) +
                                    (TZ + 1) * (TY + 1) * (TX + 1));
}

template <typename T, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) op_kernel(const cplx<T> *__restrict__ X, long sx, cplx<T> *__restrict__ Y,
                                                 long sy, const T *__restrict__ m0, const KParam *__restrict__ kp,
                                                 const int *__restrict__ act, int logN, T ih) {
  using C = cplx<T>;
  constexpr int VX = TX + 2, VY = TY + 2, VZ = TZ + 2;
  constexpr int EX = TX + 1, EY = TY + 1, EZ = TZ + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *v = reinterpret_cast<C *>(smem_raw);  // [3][VZ][VY][VX], global [o-1, o+T]
  C *e = v + 3 * VZ * VY * VX;             // [3][EZ][EY][EX], global [o, o+T]
  C *c = e + 3 * EZ * EY * EX;             // [EZ][EY][EX],    global [o-1, o+T-1]

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
  const C *Xb = X + (long)b * sx + (long)j * 3 * n;
  C *Yb = Y + (long)b * sy + (long)j * 3 * n;
  const KParam &p = kp[b];
  T kh0, kh1, kh2, gam;
  if constexpr (std::is_same<T, float>::value) {
    kh0 = p.khf[0];
    kh1 = p.khf[1];
    kh2 = p.khf[2];
    gam = p.gammaf;
  } else {
    kh0 = 0.5 * p.k[0];
    kh1 = 0.5 * p.k[1];
    kh2 = 0.5 * p.k[2];
    gam = p.gamma;
  }

  for (int i = threadIdx.x; i < 3 * VZ * VY * VX; i += blockDim.x) {
    int lx = i % VX, r = i / VX;
    int ly = r % VY;
    r /= VY;
    int lz = r % VZ, comp = r / VZ;
    int gx = (x0 + lx - 1) & mask, gy = (y0 + ly - 1) & mask, gz = (z0 + lz - 1) & mask;
    v[i] = Xb[comp * n + ((long)gz << (2 * logN)) + ((long)gy << logN) + gx];
  }
  __syncthreads();

  for (int i = threadIdx.x; i < EZ * EY * EX; i += blockDim.x) {
    const int ex = i % EX, ey = (i / EX) % EY, ez = i / (EX * EY);
    // e at global o + (ez,ey,ex): v local index + 1; its backward neighbours are local + 0
#define VV(comp, dz, dy, dx) v[(((comp) * VZ + ez + 1 + (dz)) * VY + ey + 1 + (dy)) * VX + ex + 1 + (dx)]
    const C v1 = VV(0, 0, 0, 0), v2 = VV(1, 0, 0, 0), v3 = VV(2, 0, 0, 0);
    const C d3v2 = dbwd(VV(1, -1, 0, 0), v2, ih, kh2);
    const C d2v3 = dbwd(VV(2, 0, -1, 0), v3, ih, kh1);
    const C d3v1 = dbwd(VV(0, -1, 0, 0), v1, ih, kh2);
    const C d1v3 = dbwd(VV(2, 0, 0, -1), v3, ih, kh0);
    const C d2v1 = dbwd(VV(0, 0, -1, 0), v1, ih, kh1);
    const C d1v2 = dbwd(VV(1, 0, 0, -1), v2, ih, kh0);
#undef VV
    const int gx = (x0 + ex) & mask, gy = (y0 + ey) & mask, gz = (z0 + ez) & mask;
    const long gi = ((long)gz << (2 * logN)) + ((long)gy << logN) + gx;
    const int eo = (ez * EY + ey) * EX + ex;
    e[eo] = cscale(csub(d3v2, d2v3), m0[gi]);
    e[EZ * EY * EX + eo] = cscale(csub(d1v3, d3v1), m0[n + gi]);
    e[2 * EZ * EY * EX + eo] = cscale(csub(d2v1, d1v2), m0[2 * n + gi]);
    // c at global o - 1 + (ez,ey,ex): v local index + 0; its forward neighbours are local + 1
#define WW(comp, dz, dy, dx) v[(((comp) * VZ + ez + (dz)) * VY + ey + (dy)) * VX + ex + (dx)]
    C cc = dfwd(WW(0, 0, 0, 0), WW(0, 0, 0, 1), ih, kh0);
    cc = cadd(cc, dfwd(WW(1, 0, 0, 0), WW(1, 0, 1, 0), ih, kh1));
    cc = cadd(cc, dfwd(WW(2, 0, 0, 0), WW(2, 1, 0, 0), ih, kh2));
#undef WW
    c[eo] = cc;
  }
  __syncthreads();

  for (int i = threadIdx.x; i < TZ * TY * TX; i += blockDim.x) {
    const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
#define EE(comp, dz, dy, dx) e[(((comp) * EZ + lz + (dz)) * EY + ly + (dy)) * EX + lx + (dx)]
#define CC(dz, dy, dx) c[((lz + 1 + (dz)) * EY + ly + 1 + (dy)) * EX + lx + 1 + (dx)]
    const C c0 = CC(0, 0, 0);
    const C e1 = EE(0, 0, 0, 0), e2 = EE(1, 0, 0, 0), e3 = EE(2, 0, 0, 0);
    C y1 = csub(dfwd(e3, EE(2, 0, 1, 0), ih, kh1), dfwd(e2, EE(1, 1, 0, 0), ih, kh2));
    y1 = cadd(y1, cscale(dbwd(CC(0, 0, -1), c0, ih, kh0), gam));
    C y2 = csub(dfwd(e1, EE(0, 1, 0, 0), ih, kh2), dfwd(e3, EE(2, 0, 0, 1), ih, kh0));
    y2 = cadd(y2, cscale(dbwd(CC(0, -1, 0), c0, ih, kh1), gam));
    C y3 = csub(dfwd(e2, EE(1, 0, 0, 1), ih, kh0), dfwd(e1, EE(0, 0, 1, 0), ih, kh1));
    y3 = cadd(y3, cscale(dbwd(CC(-1, 0, 0), c0, ih, kh2), gam));
#undef EE
#undef CC
    const long gi = ((long)(z0 + lz) << (2 * logN)) + ((long)(y0 + ly) << logN) + x0 + lx;
    Yb[gi] = y1;
    Yb[n + gi] = y2;
    Yb[2 * n + gi] = y3;
  }
}

// ------------------------------------------------------------------------------------------------ z-marching stencil
// The same operator with a 2.5D blocking: a block owns a TX x TY column tile and walks ZC consecutive z planes. Per
// plane z it loads v(z+1) (with a one-point x/y halo), forms e(z+1) = M0 A' v on the tile grown by one point in +x/+y
// and c(z) = B v on the tile grown by one point in -x/-y, and writes y(z) = A e + gamma B' c from the two e planes
// (z, z+1) and the two c planes (z-1, z) held in ring buffers. Halo work is (TX+1)(TY+1)/(TX TY) instead of the
// (TX+1)(TY+1)(TZ+1)/(TX TY TZ) of the cube tile, and only 2+2+2 planes live in shared memory.
template <typename T, int TX, int TY> constexpr size_t opz_smem_bytes() {
  return sizeof(cplx<T>) * (size_t)(2 * 3 * (TY + 2) * (TX + 2) + 2 * 3 * (TY + 1) * (TX + 1) + 2 * (TY + 1) * (TX + 1));
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, 6) opz_kernel(const cplx<T> *__restrict__ X, long sx, cplx<T> *__restrict__ Y,
                                                      long sy, const T *__restrict__ m0, const KParam *__restrict__ kp,
                                                      const int *__restrict__ act, int logN, int ZC, T ih) {
  using C = cplx<T>;
  constexpr int VX = TX + 2, VY = TY + 2, VP = VX * VY;  // v plane: local (lx, ly) <-> global (x0 + lx - 1, ...)
  constexpr int EX = TX + 1, EY = TY + 1, EP = EX * EY;  // e plane: global x0 + ex; c plane: global x0 + ex - 1
  constexpr int NT = TX * TY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *vbuf = reinterpret_cast<C *>(smem_raw);  // [2][3][VP]
  C *ebuf = vbuf + 2 * 3 * VP;                 // [2][3][EP]
  C *cbuf = ebuf + 2 * 3 * EP;                 // [2][EP]
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
  const C *Xb = X + (long)b * sx + (long)j * 3 * n;
  C *Yb = Y + (long)b * sy + (long)j * 3 * n;
  const KParam &p = kp[b];
  T kh0, kh1, kh2, gam;
  if constexpr (std::is_same<T, float>::value) {
    kh0 = p.khf[0];
    kh1 = p.khf[1];
    kh2 = p.khf[2];
    gam = p.gammaf;
  } else {
    kh0 = 0.5 * p.k[0];
    kh1 = 0.5 * p.k[1];
    kh2 = 0.5 * p.k[2];
    gam = p.gamma;
  }
  const int tid = threadIdx.x;
  // The plane-independent part of every index this thread uses is formed once, before the z walk (32-bit offsets:
  // a field block holds 3 N^3 <= 2^26 entries); per plane only the z offset is added.
  constexpr int NV = (3 * VP + NT - 1) / NT;  // v entries per thread and plane
  constexpr int NE = (EP + NT - 1) / NT;      // e and c entries per thread and plane
  const int pl = (int)plane, ni = (int)n;
  int voff[NV];  // global offset of v entry tid + k NT within its plane (with the component), -1 past the plane
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const int i = tid + k * NT;
    const int comp = i / VP, r = i - comp * VP, ly = r / VX, lx = r - ly * VX;
    voff[k] = i < 3 * VP ? comp * ni + (((y0 + ly - 1) & mask) << logN) + ((x0 + lx - 1) & mask) : -1;
  }
  int eoff[NE], eloc[NE];  // e entry tid + k NT: M0 offset within its plane (-1 past the tile) and v local index
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    const int i = tid + k * NT;
    const int ey = i / EX, ex = i - ey * EX;
    eoff[k] = i < EP ? (((y0 + ey) & mask) << logN) + ((x0 + ex) & mask) : -1;
    eloc[k] = (ey + 1) * VX + ex + 1;  // v local index of global (x0 + ex, y0 + ey)
  }
  const int ly = tid / TX, lx = tid - ly * TX;
  const int yoff = ((y0 + ly) << logN) + x0 + lx;  // output point within its plane
  const int eo = ly * EX + lx;                      // e index of (x0+lx, y0+ly)
  const int co = (ly + 1) * EX + lx + 1;            // c index of (x0+lx, y0+ly)

  auto load_v = [&](int slot, int z) {
    const int zo = (z & mask) * pl;
    C *vs = vbuf + slot * 3 * VP;
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (voff[k] >= 0) vs[tid + k * NT] = Xb[voff[k] + zo];
  };
  // e(z) from v(z) (slot sz) and v(z-1) (slot szm), on the tile grown by one in +x/+y
  auto make_e = [&](int eslot, int z, int sz, int szm) {
    const C *v0 = vbuf + sz * 3 * VP, *vm = vbuf + szm * 3 * VP;
    C *es = ebuf + eslot * 3 * EP;
    const int zo = (z & mask) * pl;
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      if (eoff[k] < 0) continue;
      const int i = tid + k * NT, o = eloc[k];
      const C v1 = v0[o], v2 = v0[VP + o], v3 = v0[2 * VP + o];
      const C d3v2 = dbwd(vm[VP + o], v2, ih, kh2);
      const C d2v3 = dbwd(v0[2 * VP + o - VX], v3, ih, kh1);
      const C d3v1 = dbwd(vm[o], v1, ih, kh2);
      const C d1v3 = dbwd(v0[2 * VP + o - 1], v3, ih, kh0);
      const C d2v1 = dbwd(v0[o - VX], v1, ih, kh1);
      const C d1v2 = dbwd(v0[VP + o - 1], v2, ih, kh0);
      const int gi = zo + eoff[k];
      es[i] = cscale(csub(d3v2, d2v3), m0[gi]);
      es[EP + i] = cscale(csub(d1v3, d3v1), m0[ni + gi]);
      es[2 * EP + i] = cscale(csub(d2v1, d1v2), m0[2 * ni + gi]);
    }
  };
  // c(z) from v(z) (slot sz) and v(z+1) (slot szp), on the tile grown by one in -x/-y
  auto make_c = [&](int cslot, int sz, int szp) {
    const C *v0 = vbuf + sz * 3 * VP, *vp = vbuf + szp * 3 * VP;
    C *cs = cbuf + cslot * EP;
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      if (eoff[k] < 0) continue;
      const int i = tid + k * NT, o = eloc[k] - VX - 1;  // v local index of global (x0 + cx - 1, y0 + cy - 1)
      C cc = dfwd(v0[o], v0[o + 1], ih, kh0);
      cc = cadd(cc, dfwd(v0[VP + o], v0[VP + o + VX], ih, kh1));
      cc = cadd(cc, dfwd(v0[2 * VP + o], vp[2 * VP + o], ih, kh2));
      cs[i] = cc;
    }
  };

  // prologue: v(zb-1), v(zb) -> e(zb), c(zb-1)
  load_v(0, zb - 1);
  load_v(1, zb);
  __syncthreads();
  make_e(0, zb, 1, 0);
  make_c(0, 0, 1);
  int sv = 1, se = 0, sc = 0;  // slots holding v(z), e(z), c(z-1)
  for (int z = zb; z < zb + ZC; ++z) {
    __syncthreads();                     // previous y(z-1) done reading; v(z-1) slot free
    load_v(1 - sv, z + 1);               // v(z+1) into the free slot
    __syncthreads();
    make_e(1 - se, z + 1, 1 - sv, sv);   // e(z+1)
    make_c(1 - sc, sv, 1 - sv);          // c(z)
    __syncthreads();
    {
      const C *e0 = ebuf + se * 3 * EP, *e1p = ebuf + (1 - se) * 3 * EP;  // e(z), e(z+1)
      const C *cm = cbuf + sc * EP, *c0p = cbuf + (1 - sc) * EP;          // c(z-1), c(z)
      const C c0 = c0p[co];
      const C e1 = e0[eo], e2 = e0[EP + eo], e3 = e0[2 * EP + eo];
      C y1 = csub(dfwd(e3, e0[2 * EP + eo + EX], ih, kh1), dfwd(e2, e1p[EP + eo], ih, kh2));
      y1 = cadd(y1, cscale(dbwd(c0p[co - 1], c0, ih, kh0), gam));
      C y2 = csub(dfwd(e1, e1p[eo], ih, kh2), dfwd(e3, e0[2 * EP + eo + 1], ih, kh0));
      y2 = cadd(y2, cscale(dbwd(c0p[co - EX], c0, ih, kh1), gam));
      C y3 = csub(dfwd(e2, e0[EP + eo + 1], ih, kh0), dfwd(e1, e0[eo + EX], ih, kh1));
      y3 = cadd(y3, cscale(dbwd(cm[co], c0, ih, kh2), gam));
      const int gi = z * pl + yoff;
      Yb[gi] = y1;
      Yb[ni + gi] = y2;
      Yb[2 * ni + gi] = y3;
    }
    sv = 1 - sv;
    se = 1 - se;
    sc = 1 - sc;
  }
}

// ------------------------------------------------------------------------------------------------ row-warp z march
// Complex64 Op X for N = 32 XPL (XPL = 1, 2, 4 consecutive x values per lane): one warp per grid row, so that the
// x-neighbours of every point are in the same warp (register shuffles, with the periodic wrap inside the warp), the
// z-neighbours stay in registers along the z walk, and only the y-neighbours go through shared memory. A CTA holds
// TY + 2 warps on rows y0 - 1 .. y0 + TY; warp w loads v on its row R_w = y0 - 1 + w, forms e = M0 A' v on R_w
// (w >= 1; needs v at R_w - 1) and c = B v on R_w (w <= TY; needs v at R_w + 1), and warps 1..TY write
// y = A e + gamma B' c on their rows (e at R_w + 1 and c at R_w - 1 from the neighbouring warps). Per z plane: the
// plane of v in shared memory (three components), e1 and e3 (the components needed at +y) and c, double buffered
// where a plane is read one step later; two barriers per plane.
template <int XPL> struct OpzRow {
  static constexpr int TY = 8;
  static constexpr int WARPS = TY + 2;
  static constexpr int N = 32 * XPL;
  // v [2][3][WARPS][N], e (e1, e3) [2][2][WARPS][N], c [WARPS][N]
  static constexpr size_t smem() { return sizeof(float2) * (size_t)(2 * 3 + 2 * 2 + 1) * WARPS * N; }
};

template <int XPL> __device__ __forceinline__ void ld_row(const float2 *p, float2 (&v)[XPL]) {
  if constexpr (XPL == 1) {
    v[0] = *p;
  } else {
#pragma unroll
    for (int i = 0; i < XPL; i += 2) {
      const float4 q = *reinterpret_cast<const float4 *>(p + i);
      v[i] = make_float2(q.x, q.y);
      v[i + 1] = make_float2(q.z, q.w);
    }
  }
}
template <int XPL> __device__ __forceinline__ void st_row(float2 *p, const float2 (&v)[XPL]) {
  if constexpr (XPL == 1) {
    *p = v[0];
  } else {
#pragma unroll
    for (int i = 0; i < XPL; i += 2)
      *reinterpret_cast<float4 *>(p + i) = make_float4(v[i].x, v[i].y, v[i + 1].x, v[i + 1].y);
  }
}
template <int XPL> __device__ __forceinline__ void ld_row_m0(const float *p, float (&v)[XPL]) {
  if constexpr (XPL == 1) {
    v[0] = *p;
  } else if constexpr (XPL == 2) {
    const float2 q = *reinterpret_cast<const float2 *>(p);
    v[0] = q.x;
    v[1] = q.y;
  } else {
#pragma unroll
    for (int i = 0; i < XPL; i += 4) {
      const float4 q = *reinterpret_cast<const float4 *>(p + i);
      v[i] = q.x;
      v[i + 1] = q.y;
      v[i + 2] = q.z;
      v[i + 3] = q.w;
    }
  }
}
// the value at x - 1 of each of this lane's points (the previous lane's last point for the first one, periodic)
template <int XPL> __device__ __forceinline__ void xprev(const float2 (&v)[XPL], float2 (&o)[XPL], int lane) {
  const int src = (lane + 31) & 31;
  o[0] = make_float2(__shfl_sync(0xffffffffu, v[XPL - 1].x, src), __shfl_sync(0xffffffffu, v[XPL - 1].y, src));
#pragma unroll
  for (int i = 1; i < XPL; ++i) o[i] = v[i - 1];
}
// the value at x + 1 of each of this lane's points (the next lane's first point for the last one, periodic)
template <int XPL> __device__ __forceinline__ void xnext(const float2 (&v)[XPL], float2 (&o)[XPL], int lane) {
  const int src = (lane + 1) & 31;
  o[XPL - 1] = make_float2(__shfl_sync(0xffffffffu, v[0].x, src), __shfl_sync(0xffffffffu, v[0].y, src));
#pragma unroll
  for (int i = 0; i + 1 < XPL; ++i) o[i] = v[i + 1];
}

template <int XPL>
__global__ void __launch_bounds__(OpzRow<XPL>::WARPS * 32) opz_row_kernel(const float2 *__restrict__ X, long sx,
                                                                          float2 *__restrict__ Y, long sy,
                                                                          const float *__restrict__ m0,
                                                                          const KParam *__restrict__ kp,
                                                                          const int *__restrict__ act, int ZC) {
  using CF = OpzRow<XPL>;
  constexpr int N = CF::N, TY = CF::TY, W = CF::WARPS, PL = W * N;  // PL: one component plane of the CTA's rows
  constexpr int mask = N - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *vs = reinterpret_cast<float2 *>(smem_raw);  // [2][3][W][N]
  float2 *es = vs + 2 * 3 * PL;                         // [2][2][W][N]: e1, e3
  float2 *cs = es + 2 * 2 * PL;                         // [W][N]
  const long n = (long)N * N * N, plane = (long)N * N;
  const int b = act ? act[blockIdx.z] : (int)blockIdx.z;
  const int j = blockIdx.y;
  const int tilesY = N / TY;
  const int y0 = (blockIdx.x % tilesY) * TY;
  const int zb = (blockIdx.x / tilesY) * ZC;
  const float2 *Xb = X + (long)b * sx + (long)j * 3 * n;
  float2 *Yb = Y + (long)b * sy + (long)j * 3 * n;
  const KParam &p = kp[b];
  const float kh0 = p.khf[0], kh1 = p.khf[1], kh2 = p.khf[2], gam = p.gammaf, ih = (float)N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int R = (y0 - 1 + w) & mask;
  const int x0 = lane * XPL;
  const long rowoff = (long)R * N + x0;  // within a plane
  const bool has_e = w >= 1, has_c = w <= TY, has_y = w >= 1 && w <= TY;
  float2 *const vrow0 = vs + w * N + x0;  // slot s, component c: + (3 s + c) PL
  float2 *const erow0 = es + w * N + x0;  // slot s, (e1, e3): + (2 s + 0 / 1) PL
  float2 *const crow = cs + w * N + x0;
  auto vrow = [&](int slot) { return vrow0 + slot * 3 * PL; };
  auto erow = [&](int slot) { return erow0 + slot * 2 * PL; };

  auto load_v = [&](int z, float2 (&v)[3][XPL]) {
    const long o = (long)(z & mask) * plane + rowoff;
#pragma unroll
    for (int c = 0; c < 3; ++c) ld_row<XPL>(Xb + c * n + o, v[c]);
  };
  auto store_v = [&](int slot, const float2 (&v)[3][XPL]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) st_row<XPL>(vrow(slot) + c * PL, v[c]);
  };
  auto load_m0 = [&](int z, float (&mz)[3][XPL]) {
    const long o = (long)(z & mask) * plane + rowoff;
#pragma unroll
    for (int c = 0; c < 3; ++c) ld_row_m0<XPL>(m0 + c * n + o, mz[c]);
  };
  // e = M0 A' v at plane z on this row: v (own, plane z), vm (own, plane z - 1), v at row R - 1 from slot s, mz the
  // M0 entries of the row at plane z
  auto make_e = [&](const float (&mz)[3][XPL], int s, const float2 (&v)[3][XPL], const float2 (&vm)[3][XPL],
                    float2 (&e)[3][XPL]) {
    float2 v1y[XPL], v3y[XPL], v2x[XPL], v3x[XPL];
    ld_row<XPL>(vrow(s) - N, v1y);           // v1 at R - 1
    ld_row<XPL>(vrow(s) + 2 * PL - N, v3y);  // v3 at R - 1
    xprev<XPL>(v[1], v2x, lane);
    xprev<XPL>(v[2], v3x, lane);
#pragma unroll
    for (int i = 0; i < XPL; ++i) {
      const float2 d3v2 = dbwd(vm[1][i], v[1][i], ih, kh2), d2v3 = dbwd(v3y[i], v[2][i], ih, kh1);
      const float2 d3v1 = dbwd(vm[0][i], v[0][i], ih, kh2), d1v3 = dbwd(v3x[i], v[2][i], ih, kh0);
      const float2 d2v1 = dbwd(v1y[i], v[0][i], ih, kh1), d1v2 = dbwd(v2x[i], v[1][i], ih, kh0);
      e[0][i] = cscale(csub(d3v2, d2v3), mz[0][i]);
      e[1][i] = cscale(csub(d1v3, d3v1), mz[1][i]);
      e[2][i] = cscale(csub(d2v1, d1v2), mz[2][i]);
    }
  };
  // c = B v at plane z on this row: v (own, plane z), v2 at R + 1 from slot s (plane z), v3 of plane z + 1 (own)
  auto make_c = [&](int s, const float2 (&v)[3][XPL], const float2 (&vp3)[XPL], float2 (&cc)[XPL]) {
    float2 v2y[XPL], v1x[XPL];
    ld_row<XPL>(vrow(s) + PL + N, v2y);  // v2 at R + 1
    xnext<XPL>(v[0], v1x, lane);
#pragma unroll
    for (int i = 0; i < XPL; ++i)
      cc[i] = cadd(cadd(dfwd(v[0][i], v1x[i], ih, kh0), dfwd(v[1][i], v2y[i], ih, kh1)),
                   dfwd(v[2][i], vp3[i], ih, kh2));
  };

  float2 vm[3][XPL], v0[3][XPL], vp[3][XPL], ecur[3][XPL], enext[3][XPL], cprev[XPL], ccur[XPL];
  // (the edge warps shuffle values they never use: start them defined)
#pragma unroll
  for (int i = 0; i < XPL; ++i) {
    cprev[i] = ccur[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) ecur[c][i] = enext[c][i] = make_float2(0.f, 0.f);
  }
  // prologue: v(zb - 1) into slot 1, v(zb) into slot 0; c(zb - 1) and e(zb)
  load_v(zb - 1, vm);
  load_v(zb, v0);
  store_v(1, vm);
  store_v(0, v0);
  __syncthreads();
  if (has_c) make_c(1, vm, v0[2], cprev);
  if (has_e) {
    float mz0[3][XPL];
    load_m0(zb, mz0);
    make_e(mz0, 0, v0, vm, ecur);
    st_row<XPL>(erow(0), ecur[0]);
    st_row<XPL>(erow(0) + PL, ecur[2]);
  }
  __syncthreads();  // slot 1 (v(zb - 1)) is rewritten by the first step
  int s0 = 0, es0 = 0;  // slots of v(z) and e(z)
  // v of the next plane is loaded one step ahead (vn), so that its latency overlaps a whole step
  float2 vn[3][XPL];
  float mn[3][XPL], mz[3][XPL];
  load_v(zb + 1, vn);
  load_m0(zb + 1, mn);
  for (int z = zb; z < zb + ZC; ++z) {
    const int s1 = 1 - s0, es1 = 1 - es0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int i = 0; i < XPL; ++i) {
        vp[c][i] = vn[c][i];
        mz[c][i] = mn[c][i];
      }
    if (z + 1 < zb + ZC) {
      load_v(z + 2, vn);
      load_m0(z + 2, mn);
    }
    store_v(s1, vp);  // slot s1 held v(z - 1): its last readers (c(z - 1)) finished before the previous barrier
    __syncthreads();
    if (has_e) {
      make_e(mz, s1, vp, v0, enext);
      st_row<XPL>(erow(es1), enext[0]);
      st_row<XPL>(erow(es1) + PL, enext[2]);
    }
    if (has_c) {
      make_c(s0, v0, vp[2], ccur);
      st_row<XPL>(crow, ccur);
    }
    __syncthreads();
    // every warp takes part in the shuffles; warps 0 and TY + 1 hold no output row
    float2 e3x[XPL], e2x[XPL], cx[XPL];
    xnext<XPL>(ecur[2], e3x, lane);
    xnext<XPL>(ecur[1], e2x, lane);
    xprev<XPL>(ccur, cx, lane);
    if (has_y) {
      float2 e1y[XPL], e3y[XPL], cy[XPL];
      ld_row<XPL>(erow(es0) + N, e1y);       // e1(z) at R + 1
      ld_row<XPL>(erow(es0) + PL + N, e3y);  // e3(z) at R + 1
      ld_row<XPL>(crow - N, cy);             // c(z) at R - 1
      float2 o1[XPL], o2[XPL], o3[XPL];
#pragma unroll
      for (int i = 0; i < XPL; ++i) {
        const float2 e1 = ecur[0][i], e2 = ecur[1][i], e3 = ecur[2][i], c0 = ccur[i];
        o1[i] = cadd(csub(dfwd(e3, e3y[i], ih, kh1), dfwd(e2, enext[1][i], ih, kh2)),
                     cscale(dbwd(cx[i], c0, ih, kh0), gam));
        o2[i] = cadd(csub(dfwd(e1, enext[0][i], ih, kh2), dfwd(e3, e3x[i], ih, kh0)),
                     cscale(dbwd(cy[i], c0, ih, kh1), gam));
        o3[i] = cadd(csub(dfwd(e2, e2x[i], ih, kh0), dfwd(e1, e1y[i], ih, kh1)),
                     cscale(dbwd(cprev[i], c0, ih, kh2), gam));
      }
      const long o = (long)z * plane + rowoff;
      st_row<XPL>(Yb + o, o1);
      st_row<XPL>(Yb + n + o, o2);
      st_row<XPL>(Yb + 2 * n + o, o3);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int i = 0; i < XPL; ++i) {
        vm[c][i] = v0[c][i];
        v0[c][i] = vp[c][i];
        ecur[c][i] = enext[c][i];
      }
#pragma unroll
    for (int i = 0; i < XPL; ++i) cprev[i] = ccur[i];
    s0 = s1;
    es0 = es1;
  }
}

// ------------------------------------------------------------------------------------------------ half applies
// A' x at edge point r and B x at cell point r, read straight from global memory (not on the per-iteration path).
struct HalfOut {
  double2 e[3];
  double2 c;
};
// S: complex128 (double2) or double-float pairs (float4), read as FP64 values
template <typename S>
__device__ __forceinline__ HalfOut half_at(const S *__restrict__ x, long n, int logN, int gx, int gy, int gz,
                                           double ih, double kh0, double kh1, double kh2) {
  const int mask = (1 << logN) - 1;
  auto at = [&](int comp, int z, int y, int xx) {
    return ld_c128(x + comp * n + ((long)(z & mask) << (2 * logN)) + ((long)(y & mask) << logN) + (xx & mask));
  };
  const double2 v1 = at(0, gz, gy, gx), v2 = at(1, gz, gy, gx), v3 = at(2, gz, gy, gx);
  HalfOut o;
  o.e[0] = csub(dbwd(at(1, gz - 1, gy, gx), v2, ih, kh2), dbwd(at(2, gz, gy - 1, gx), v3, ih, kh1));
  o.e[1] = csub(dbwd(at(2, gz, gy, gx - 1), v3, ih, kh0), dbwd(at(0, gz - 1, gy, gx), v1, ih, kh2));
  o.e[2] = csub(dbwd(at(0, gz, gy - 1, gx), v1, ih, kh1), dbwd(at(1, gz, gy, gx - 1), v2, ih, kh0));
  o.c = cadd(cadd(dfwd(v1, at(0, gz, gy, gx + 1), ih, kh0), dfwd(v2, at(1, gz, gy + 1, gx), ih, kh1)),
             dfwd(v3, at(2, gz + 1, gy, gx), ih, kh2));
  return o;
}

__global__ void half_kernel(const double2 *__restrict__ X, double2 *__restrict__ E, double2 *__restrict__ Cc,
                            const KParam *__restrict__ kp, int logN, int m, double ih) {
  const long n = 1L << (3 * logN);
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = blockIdx.z, j = blockIdx.y;
  const int N = 1 << logN;
  const int gx = (int)(i & (N - 1)), gy = (int)((i >> logN) & (N - 1)), gz = (int)(i >> (2 * logN));
  const KParam p = kp[b];
  const double2 *x = X + ((long)b * m + j) * 3 * n;
  HalfOut o = half_at(x, n, logN, gx, gy, gz, ih, 0.5 * p.k[0], 0.5 * p.k[1], 0.5 * p.k[2]);
  if (E) {
    double2 *eb = E + ((long)b * m + j) * 3 * n;
    eb[i] = o.e[0];
    eb[n + i] = o.e[1];
    eb[2 * n + i] = o.e[2];
  }
  if (Cc) Cc[((long)b * m + j) * n + i] = o.c;
}

// per-block partial sums of (sum M0 |A'x|^2, sum |Bx|^2, sum |x|^2); grid (nchunk, m, nb)
template <typename S>
__global__ void recompute_partial_kernel(const S *__restrict__ X, long sx, const double *__restrict__ m0,
                                         const KParam *__restrict__ kp, const int *__restrict__ act, int logN,
                                         double ih, long chunk, double *__restrict__ part) {
  const long n = 1L << (3 * logN);
  const int N = 1 << logN;
  const int bi = blockIdx.z;
  const int b = act ? act[bi] : bi;
  const int j = blockIdx.y;
  const KParam p = kp[b];
  const S *x = X + (long)b * sx + (long)j * 3 * n;
  double s0 = 0, s1 = 0, s2 = 0;
  const long beg = blockIdx.x * chunk, end = min(n, beg + chunk);
  for (long i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const int gx = (int)(i & (N - 1)), gy = (int)((i >> logN) & (N - 1)), gz = (int)(i >> (2 * logN));
    HalfOut o = half_at(x, n, logN, gx, gy, gz, ih, 0.5 * p.k[0], 0.5 * p.k[1], 0.5 * p.k[2]);
    for (int c = 0; c < 3; ++c) {
      s0 += m0[c * n + i] * (o.e[c].x * o.e[c].x + o.e[c].y * o.e[c].y);
      const double2 xv = ld_c128(x + c * n + i);
      s2 += xv.x * xv.x + xv.y * xv.y;
    }
    s1 += o.c.x * o.c.x + o.c.y * o.c.y;
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double *o = part + (((long)bi * gridDim.y + j) * gridDim.x + blockIdx.x) * 3;
    o[0] = red[0][0];
    o[1] = red[1][0];
    o[2] = red[2][0];
  }
}

__global__ void recompute_reduce_kernel(const double *__restrict__ part, int nchunk, int m,
                                        const int *__restrict__ act, double *__restrict__ out) {
  const int bi = blockIdx.x, j = threadIdx.x;
  if (j >= m) return;
  const int b = act ? act[bi] : bi;
  double s[3] = {0, 0, 0};
  for (int c = 0; c < nchunk; ++c)
    for (int q = 0; q < 3; ++q) s[q] += part[(((long)bi * m + j) * nchunk + c) * 3 + q];
  for (int q = 0; q < 3; ++q) out[((long)b * m + j) * 3 + q] = s[q];
}

// ------------------------------------------------------------------------------------------------ launchers
template <typename T, int TX, int TY, int TZ>
static int launch_op_t(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act) {
  constexpr size_t smem = op_smem_bytes<T, TX, TY, TZ>();
  static bool configured = false;  // attribute is per function; set once per process
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(op_kernel<T, TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  const int N = ctx->N;
  dim3 grid((N / TX) * (N / TY) * (N / TZ), m, nb);
  const T *m0 = std::is_same<T, double>::value ? ctx->m0d.as<T>() : ctx->m0f.as<T>();
  op_kernel<T, TX, TY, TZ><<<grid, 256, smem, ctx->stream>>>(
      static_cast<const cplx<T> *>(X), sx, static_cast<cplx<T> *>(Y), sy, m0, ctx->kparam.as<KParam>(), act,
      ctx->logN, (T)ctx->N);
  PC_CK_LAUNCH();
  return PC_OK;
}

template <typename T, int TX, int TY>
static int launch_opz_t(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act) {
  constexpr size_t smem = opz_smem_bytes<T, TX, TY>();
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(opz_kernel<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  const int N = ctx->N;
  // z chunk: enough blocks to fill the GPU several times over, at least 4 planes per chunk
  const long tiles = (long)(N / TX) * (N / TY) * m * nb;
  int ZC = N;
  while (ZC > 4 && tiles * (N / ZC) < 16L * sm_count()) ZC >>= 1;
  dim3 grid((N / TX) * (N / TY) * (N / ZC), m, nb);
  const T *m0 = std::is_same<T, double>::value ? ctx->m0d.as<T>() : ctx->m0f.as<T>();
  opz_kernel<T, TX, TY><<<grid, TX * TY, smem, ctx->stream>>>(static_cast<const cplx<T> *>(X), sx,
                                                                static_cast<cplx<T> *>(Y), sy, m0,
                                                                ctx->kparam.as<KParam>(), act, ctx->logN, ZC, (T)ctx->N);
  PC_CK_LAUNCH();
  return PC_OK;
}

template <int XPL>
static int launch_opz_row(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act) {
  using CF = OpzRow<XPL>;
  constexpr size_t smem = CF::smem();
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(opz_row_kernel<XPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  constexpr int N = CF::N;
  // z chunk: at least about 8 CTAs per SM over the launch, at least 8 planes per chunk (the prologue loads one
  // extra plane per chunk)
  const long tiles = (long)(N / CF::TY) * m * nb;
  int ZC = N;
  while (ZC > 8 && tiles * (N / ZC) < 8L * sm_count()) ZC >>= 1;
  dim3 grid((N / CF::TY) * (N / ZC), m, nb);
  opz_row_kernel<XPL><<<grid, CF::WARPS * 32, smem, ctx->stream>>>(static_cast<const float2 *>(X), sx,
                                                                    static_cast<float2 *>(Y), sy, ctx->m0f.as<float>(),
                                                                    ctx->kparam.as<KParam>(), act, ZC);
  PC_CK_LAUNCH();
  return PC_OK;
}

int launch_apply_op(pc_ctx *ctx, int nb, int m, int dtype, const void *X, long sx, void *Y, long sy,
                    const int *act) {
  if (nb == 0 || m == 0) return PC_OK;
  if (ctx->opts.order > 1 || ctx->lat) return launch_apply_op_k(ctx, nb, m, dtype, X, sx, Y, sy, act);
  const int N = ctx->N;
  if (dtype == PC_C64 && N == 32) return launch_opz_row<1>(ctx, nb, m, X, sx, Y, sy, act);
  if (dtype == PC_C64 && N == 64) return launch_opz_row<2>(ctx, nb, m, X, sx, Y, sy, act);
  if (dtype == PC_C64 && N == 128) return launch_opz_row<4>(ctx, nb, m, X, sx, Y, sy, act);
  if (dtype == PC_C64 && N >= 32) return launch_opz_t<float, 32, 8>(ctx, nb, m, X, sx, Y, sy, act);
  if (dtype == PC_C128) {
    if (N >= 32) return launch_op_t<double, 32, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
    if (N == 16) return launch_op_t<double, 16, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
    return launch_op_t<double, 8, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
  }
  if (N >= 32) return launch_op_t<float, 32, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
  if (N == 16) return launch_op_t<float, 16, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
  return launch_op_t<float, 8, 4, 4>(ctx, nb, m, X, sx, Y, sy, act);
}

size_t recompute_scratch_bytes(long n, int nb, int m) {
  const int nchunk = (int)std::min<long>(64, (n + 4095) / 4096);
  return sizeof(double) * 3 * (size_t)nb * m * nchunk;
}

int launch_recompute(pc_ctx *ctx, int nb, int m, const void *X, long sx, double *out, const int *act, void *scratch,
                     size_t scratch_bytes, int dtype) {
  if (nb == 0 || m == 0) return PC_OK;
  const long n = ctx->n;
  const int nchunk = (int)std::min<long>(64, (n + 4095) / 4096);
  const long chunk = (n + nchunk - 1) / nchunk;
  if (recompute_scratch_bytes(n, nb, m) > scratch_bytes) {
    set_error("recompute: scratch too small");
    return PC_EINVAL;
  }
  double *part = static_cast<double *>(scratch);
  if (ctx->opts.order > 1 || ctx->lat) {
    int rc = launch_recompute_k_partial(ctx, nb, m, X, sx, act, nchunk, chunk, part, dtype);
    if (rc) return rc;
  } else if (dtype == PC_DFS)
    recompute_partial_kernel<float4><<<dim3(nchunk, m, nb), 256, 0, ctx->stream>>>(
        static_cast<const float4 *>(X), sx, ctx->m0d.as<double>(), ctx->kparam.as<KParam>(), act, ctx->logN,
        (double)ctx->N, chunk, part);
  else
    recompute_partial_kernel<double2><<<dim3(nchunk, m, nb), 256, 0, ctx->stream>>>(
        static_cast<const double2 *>(X), sx, ctx->m0d.as<double>(), ctx->kparam.as<KParam>(), act, ctx->logN,
        (double)ctx->N, chunk, part);
  PC_CK_LAUNCH();
  recompute_reduce_kernel<<<nb, 64, 0, ctx->stream>>>(part, nchunk, m, act, out);
  PC_CK_LAUNCH();
  return PC_OK;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_apply_op(pc_ctx *ctx, int nb, const double *kpts, const double *gammas, int m, int dtype,
                           const void *X, void *Y) {
  PC_REQUIRE(ctx && kpts && gammas && X && Y, "pc_apply_op: null argument");
  PC_REQUIRE(nb >= 0 && m >= 0, "pc_apply_op: negative size");
  PC_REQUIRE(dtype == PC_C128 || dtype == PC_C64 || dtype == PC_C128_DF, "pc_apply_op: bad dtype %d", dtype);
  int rc = upload_kpoints(ctx, nb, kpts, gammas);
  if (rc) return rc;
  const long blk = (long)m * 3 * ctx->n;
  if (dtype == PC_C128_DF) return launch_apply_op_df(ctx, nb, m, X, blk, Y, blk, nullptr);
  return launch_apply_op(ctx, nb, m, dtype, X, blk, Y, blk, nullptr);
}

extern "C" int pc_apply_half(pc_ctx *ctx, int nb, const double *kpts, int m, const void *X, void *E, void *C) {
  PC_REQUIRE(ctx && kpts && X, "pc_apply_half: null argument");
  PC_REQUIRE(nb >= 0 && m >= 0, "pc_apply_half: negative size");
  if (nb == 0 || m == 0) return PC_OK;
  std::vector<double> g(nb, 1.0);
  int rc = upload_kpoints(ctx, nb, kpts, g.data());
  if (rc) return rc;
  if (ctx->opts.order > 1 || ctx->lat) return launch_half_k(ctx, nb, m, X, E, C);
  dim3 grid((unsigned)((ctx->n + 255) / 256), m, nb);
  half_kernel<<<grid, 256, 0, ctx->stream>>>(static_cast<const double2 *>(X), static_cast<double2 *>(E),
                                              static_cast<double2 *>(C), ctx->kparam.as<KParam>(), ctx->logN, m,
                                              (double)ctx->N);
  PC_CK_LAUNCH();
  return PC_OK;
}

extern "C" int pc_recompute_norms(pc_ctx *ctx, int nb, const double *kpts, int m, const void *X, double *out) {
  PC_REQUIRE(ctx && kpts && X && out, "pc_recompute_norms: null argument");
  PC_REQUIRE(nb >= 0 && m >= 0 && m <= 64, "pc_recompute_norms: bad size");
  std::vector<double> g(nb, 1.0);
  int rc = upload_kpoints(ctx, nb, kpts, g.data());
  if (rc) return rc;
  PC_CK(ctx->scratch.reserve(recompute_scratch_bytes(ctx->n, nb, m)));
  return launch_recompute(ctx, nb, m, X, (long)m * 3 * ctx->n, out, nullptr, ctx->scratch.p, ctx->scratch.bytes);
}
