// Permittivity at the edge DoFs from a list of dielectric spheres (Section 4.4), one thread per edge.
// x-edge (i,j,k) sits at ((i+1/2)h, jh, kh), y-edge at (ih, (j+1/2)h, kh), z-edge at (ih, jh, (k+1/2)h); cells at
// ((i+1/2)h, (j+1/2)h, (k+1/2)h). A point is inside a sphere when its distance to the nearest periodic image of the
// centre is <= r; later spheres take precedence. An edge within 1e-12 of a sphere surface takes the interface rule
// eps = (sum of eps at the 4 cell centres sharing the edge) / 4, i.e. M0 = 4 / sum (harmonic rule of Section 4.4).
// Arithmetic uses explicit round-to-nearest intrinsics (no fused multiply-add) so that the classification of a
// point does not depend on instruction selection.
#include <cmath>
#include <vector>

#include "pc_internal.cuh"

namespace pc {

constexpr double IFACE_TOL = 1e-12;

__device__ double sphere_dist(double px, double py, double pz, const double *s) {
  double dx = __dsub_rn(px, s[0]), dy = __dsub_rn(py, s[1]), dz = __dsub_rn(pz, s[2]);
  dx = __dsub_rn(dx, rint(dx));
  dy = __dsub_rn(dy, rint(dy));
  dz = __dsub_rn(dz, rint(dz));
  return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__device__ double eps_point(double px, double py, double pz, const double *sph, int nsph, double eps_bg,
                            bool *iface) {
  double e = eps_bg;
  bool on = false;
  for (int s = 0; s < nsph; ++s) {
    const double *sp = sph + 5 * s;
    const double d = sphere_dist(px, py, pz, sp);
    if (d <= sp[3]) e = sp[4];
    if (fabs(__dsub_rn(d, sp[3])) < IFACE_TOL) on = true;
  }
  if (iface) *iface = on;
  return e;
}

__global__ void eps_edges_kernel(const double *__restrict__ sph, int nsph, double eps_bg, int N, double *out) {
  const long n = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 3 * n) return;
  const int axis = (int)(gid / n);
  const long r = gid - (long)axis * n;
  const int ix = (int)(r % N), iy = (int)((r / N) % N), iz = (int)(r / ((long)N * N));
  const double h = 1.0 / (double)N;
  double p[3] = {__dmul_rn((double)ix, h), __dmul_rn((double)iy, h), __dmul_rn((double)iz, h)};
  p[axis] = __dadd_rn(p[axis], __dmul_rn(0.5, h));
  bool on = false;
  double e = eps_point(p[0], p[1], p[2], sph, nsph, eps_bg, &on);
  if (on) {
    int o1 = (axis + 1) % 3, o2 = (axis + 2) % 3;
    if (o1 > o2) {
      const int t = o1;
      o1 = o2;
      o2 = t;
    }
    double total = 0.0;
    for (int a = -1; a <= 0; ++a)
      for (int c = -1; c <= 0; ++c) {
        int idx[3] = {ix, iy, iz};
        idx[o1] += a;
        idx[o2] += c;
        double q[3];
        for (int d = 0; d < 3; ++d) q[d] = __dmul_rn(__dadd_rn((double)idx[d], 0.5), h);
        total = __dadd_rn(total, eps_point(q[0], q[1], q[2], sph, nsph, eps_bg, nullptr));
      }
    e = total / 4.0;
  }
  out[gid] = e;
}

// ---------------------------------------------------------------------------------------------- general lattice
// Section 2's coordinate change x = A y: the grid above lives in y on the unit cube, and a DoF at y sits at the
// Cartesian point x = A y. Sphere centres and radii are Cartesian; the distance to a centre c is the minimum over its
// images c + A n, found by reducing the fractional offset A^{-1}(x - c) to [-1/2, 1/2]^3 and searching the 27
// neighbouring translates.
struct LatMat {
  double a[9], ai[9];  // A and A^{-1}, row-major
};

__device__ __forceinline__ double dot3_rn(const double *r, double v0, double v1, double v2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(r[0], v0), __dmul_rn(r[1], v1)), __dmul_rn(r[2], v2));
}

__device__ double sphere_dist_lat(const double *x, const double *s, const LatMat &L) {
  const double d0 = __dsub_rn(x[0], s[0]), d1 = __dsub_rn(x[1], s[1]), d2 = __dsub_rn(x[2], s[2]);
  double f[3];
  for (int i = 0; i < 3; ++i) {
    f[i] = dot3_rn(L.ai + 3 * i, d0, d1, d2);
    f[i] = __dsub_rn(f[i], rint(f[i]));
  }
  double best = INFINITY;
  for (int t = 0; t < 27; ++t) {
    const double g0 = __dadd_rn(f[0], (double)(t % 3 - 1)), g1 = __dadd_rn(f[1], (double)((t / 3) % 3 - 1)),
                 g2 = __dadd_rn(f[2], (double)(t / 9 - 1));
    const double v0 = dot3_rn(L.a, g0, g1, g2), v1 = dot3_rn(L.a + 3, g0, g1, g2), v2 = dot3_rn(L.a + 6, g0, g1, g2);
    best = fmin(best, sqrt(__dadd_rn(__dadd_rn(__dmul_rn(v0, v0), __dmul_rn(v1, v1)), __dmul_rn(v2, v2))));
  }
  return best;
}

__device__ double eps_point_lat(const double *y, const double *sph, int nsph, double eps_bg, const LatMat &L,
                                bool *iface) {
  const double x[3] = {dot3_rn(L.a, y[0], y[1], y[2]), dot3_rn(L.a + 3, y[0], y[1], y[2]),
                       dot3_rn(L.a + 6, y[0], y[1], y[2])};
  double e = eps_bg;
  bool on = false;
  for (int s = 0; s < nsph; ++s) {
    const double *sp = sph + 5 * s;
    const double d = sphere_dist_lat(x, sp, L);
    if (d <= sp[3]) e = sp[4];
    if (fabs(__dsub_rn(d, sp[3])) < IFACE_TOL) on = true;
  }
  if (iface) *iface = on;
  return e;
}

__global__ void eps_edges_lat_kernel(const double *__restrict__ sph, int nsph, double eps_bg, int N, const LatMat L,
                                     double *out) {
  const long n = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 3 * n) return;
  const int axis = (int)(gid / n);
  const long r = gid - (long)axis * n;
  const int ix = (int)(r % N), iy = (int)((r / N) % N), iz = (int)(r / ((long)N * N));
  const double h = 1.0 / (double)N;
  double p[3] = {__dmul_rn((double)ix, h), __dmul_rn((double)iy, h), __dmul_rn((double)iz, h)};
  p[axis] = __dadd_rn(p[axis], __dmul_rn(0.5, h));
  bool on = false;
  double e = eps_point_lat(p, sph, nsph, eps_bg, L, &on);
  if (on) {
    int o1 = (axis + 1) % 3, o2 = (axis + 2) % 3;
    if (o1 > o2) {
      const int t = o1;
      o1 = o2;
      o2 = t;
    }
    double total = 0.0;
    for (int a = -1; a <= 0; ++a)
      for (int c = -1; c <= 0; ++c) {
        int idx[3] = {ix, iy, iz};
        idx[o1] += a;
        idx[o2] += c;
        double q[3];
        for (int d = 0; d < 3; ++d) q[d] = __dmul_rn(__dadd_rn((double)idx[d], 0.5), h);
        total = __dadd_rn(total, eps_point_lat(q, sph, nsph, eps_bg, L, nullptr));
      }
    e = total / 4.0;
  }
  out[gid] = e;
}

// ------------------------------------------------------------------------------------ the structures of Section 6.3
// The BCC single gyroid {g > t}, g = sin(2 pi x / l) cos(2 pi y / l) + sin(2 pi y / l) cos(2 pi z / l)
// + sin(2 pi z / l) cos(2 pi x / l) at the Cartesian point A y of each edge midpoint (strict inequality; no interface
// rule for a level set).
__global__ void eps_gyroid_kernel(int N, const LatMat L, double l, double t, double eps_in, double eps_out,
                                  double *out) {
  const long n = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 3 * n) return;
  const int axis = (int)(gid / n);
  const long r = gid - (long)axis * n;
  const int ix = (int)(r % N), iy = (int)((r / N) % N), iz = (int)(r / ((long)N * N));
  const double h = 1.0 / (double)N;
  double p[3] = {__dmul_rn((double)ix, h), __dmul_rn((double)iy, h), __dmul_rn((double)iz, h)};
  p[axis] = __dadd_rn(p[axis], __dmul_rn(0.5, h));
  const double w = 2.0 * M_PI / l;
  double sn[3], cs[3];
  for (int i = 0; i < 3; ++i) sincos(w * dot3_rn(L.a + 3 * i, p[0], p[1], p[2]), &sn[i], &cs[i]);
  const double g = sn[0] * cs[1] + sn[1] * cs[2] + sn[2] * cs[0];
  out[gid] = g > t ? eps_in : eps_out;
}

// x - (c + A n) for the image of c nearest to x (the search of sphere_dist_lat)
__device__ void nearest_offset_lat(const double *x, const double *c, const LatMat &L, double *off) {
  const double d0 = __dsub_rn(x[0], c[0]), d1 = __dsub_rn(x[1], c[1]), d2 = __dsub_rn(x[2], c[2]);
  double f[3];
  for (int i = 0; i < 3; ++i) {
    f[i] = dot3_rn(L.ai + 3 * i, d0, d1, d2);
    f[i] = __dsub_rn(f[i], rint(f[i]));
  }
  double best = INFINITY;
  for (int t = 0; t < 27; ++t) {
    const double g0 = __dadd_rn(f[0], (double)(t % 3 - 1)), g1 = __dadd_rn(f[1], (double)((t / 3) % 3 - 1)),
                 g2 = __dadd_rn(f[2], (double)(t / 9 - 1));
    const double v0 = dot3_rn(L.a, g0, g1, g2), v1 = dot3_rn(L.a + 3, g0, g1, g2), v2 = dot3_rn(L.a + 6, g0, g1, g2);
    const double d = __dadd_rn(__dadd_rn(__dmul_rn(v0, v0), __dmul_rn(v1, v1)), __dmul_rn(v2, v2));
    if (d < best) {
      best = d;
      off[0] = v0;
      off[1] = v1;
      off[2] = v2;
    }
  }
}

// The FCC diamond: spheres of radius r l at (0, 0, 0) and (l/4)(1, 1, 1), and spheroids along the four bonds
// (l/4)(1, 1, 1), (l/4)(1, -1, -1), (l/4)(-1, 1, -1), (l/4)(-1, -1, 1) from the origin, with foci at the bond's ends
// and minor axis b l (semi-major sqrt(c^2 + (b l / 2)^2), c half the bond length); closed sets.
__global__ void eps_diamond_kernel(int N, const LatMat L, double l, double rad, double semi_major, double eps_in,
                                   double eps_out, double *out) {
  const long n = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 3 * n) return;
  const int axis = (int)(gid / n);
  const long r = gid - (long)axis * n;
  const int ix = (int)(r % N), iy = (int)((r / N) % N), iz = (int)(r / ((long)N * N));
  const double h = 1.0 / (double)N;
  double p[3] = {__dmul_rn((double)ix, h), __dmul_rn((double)iy, h), __dmul_rn((double)iz, h)};
  p[axis] = __dadd_rn(p[axis], __dmul_rn(0.5, h));
  const double x[3] = {dot3_rn(L.a, p[0], p[1], p[2]), dot3_rn(L.a + 3, p[0], p[1], p[2]),
                       dot3_rn(L.a + 6, p[0], p[1], p[2])};
  const double q = 0.25 * l;
  const double sites[2][3] = {{0.0, 0.0, 0.0}, {q, q, q}};
  const double bonds[4][3] = {{q, q, q}, {q, -q, -q}, {-q, q, -q}, {-q, -q, q}};
  bool inside = false;
  double v[3];
  for (int s = 0; s < 2 && !inside; ++s) {
    nearest_offset_lat(x, sites[s], L, v);
    inside = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) <= rad;
  }
  for (int k = 0; k < 4 && !inside; ++k) {
    const double mid[3] = {0.5 * bonds[k][0], 0.5 * bonds[k][1], 0.5 * bonds[k][2]};
    nearest_offset_lat(x, mid, L, v);
    double a2 = 0.0, b2 = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double hp = v[i] + mid[i], hm = v[i] - mid[i];  // to the two foci, at mid -/+ (bond / 2)
      a2 += hp * hp;
      b2 += hm * hm;
    }
    inside = sqrt(a2) + sqrt(b2) <= 2.0 * semi_major;
  }
  out[gid] = inside ? eps_in : eps_out;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_eps_spheres(int N, int nsph, const double *spheres, double eps_bg, double *eps_out) {
  PC_REQUIRE(eps_out && (nsph == 0 || spheres), "pc_eps_spheres: null argument");
  PC_REQUIRE(N >= 2 && N <= 1024 && nsph >= 0 && nsph <= 4096, "pc_eps_spheres: bad sizes");
  PC_REQUIRE(eps_bg > 0.0, "pc_eps_spheres: eps_bg must be > 0");
  for (int s = 0; s < nsph; ++s) PC_REQUIRE(spheres[5 * s + 4] > 0.0 && spheres[5 * s + 3] >= 0.0, "pc_eps_spheres: bad sphere %d", s);
  const long total = 3L * N * N * N;
  DevBuf ds, dout;
  PC_CK(ds.reserve(sizeof(double) * 5 * std::max(nsph, 1)));
  PC_CK(dout.reserve(sizeof(double) * total));
  if (nsph) PC_CK(cudaMemcpy(ds.p, spheres, sizeof(double) * 5 * nsph, cudaMemcpyHostToDevice));
  eps_edges_kernel<<<(unsigned)((total + 255) / 256), 256>>>(ds.as<double>(), nsph, eps_bg, N, dout.as<double>());
  PC_CK_LAUNCH();
  PC_CK(cudaMemcpy(eps_out, dout.p, sizeof(double) * total, cudaMemcpyDeviceToHost));
  return PC_OK;
}

extern "C" int pc_eps_spheres_lattice(int N, const double *lattice, int nsph, const double *spheres, double eps_bg,
                                      double *eps_out) {
  PC_REQUIRE(lattice && eps_out && (nsph == 0 || spheres), "pc_eps_spheres_lattice: null argument");
  PC_REQUIRE(N >= 2 && N <= 1024 && nsph >= 0 && nsph <= 4096, "pc_eps_spheres_lattice: bad sizes");
  PC_REQUIRE(eps_bg > 0.0, "pc_eps_spheres_lattice: eps_bg must be > 0");
  for (int i = 0; i < 9; ++i) PC_REQUIRE(std::isfinite(lattice[i]), "pc_eps_spheres_lattice: lattice not finite");
  for (int s = 0; s < nsph; ++s)
    PC_REQUIRE(spheres[5 * s + 4] > 0.0 && spheres[5 * s + 3] >= 0.0, "pc_eps_spheres_lattice: bad sphere %d", s);
  LatMat L;
  if (invert_lattice(lattice, L.a, L.ai) != 0) {
    set_error("pc_eps_spheres_lattice: the lattice vectors must be linearly independent");
    return PC_EINVAL;
  }
  const long total = 3L * N * N * N;
  DevBuf ds, dout;
  PC_CK(ds.reserve(sizeof(double) * 5 * std::max(nsph, 1)));
  PC_CK(dout.reserve(sizeof(double) * total));
  if (nsph) PC_CK(cudaMemcpy(ds.p, spheres, sizeof(double) * 5 * nsph, cudaMemcpyHostToDevice));
  eps_edges_lat_kernel<<<(unsigned)((total + 255) / 256), 256>>>(ds.as<double>(), nsph, eps_bg, N, L,
                                                                 dout.as<double>());
  PC_CK_LAUNCH();
  PC_CK(cudaMemcpy(eps_out, dout.p, sizeof(double) * total, cudaMemcpyDeviceToHost));
  return PC_OK;
}

namespace {

int eps_structure_common(const char *who, int N, const double *lattice, double *eps_out, LatMat *L) {
  PC_REQUIRE(lattice && eps_out, "%s: null argument", who);
  PC_REQUIRE(N >= 2 && N <= 1024, "%s: bad N %d", who, N);
  for (int i = 0; i < 9; ++i) PC_REQUIRE(std::isfinite(lattice[i]), "%s: lattice not finite", who);
  if (invert_lattice(lattice, L->a, L->ai) != 0) {
    set_error("%s: the lattice vectors must be linearly independent", who);
    return PC_EINVAL;
  }
  return PC_OK;
}

}  // namespace

extern "C" int pc_eps_gyroid(int N, const double *lattice, double l, double threshold, double eps_in, double eps_bg,
                             double *eps_out) {
  LatMat L;
  int rc = eps_structure_common("pc_eps_gyroid", N, lattice, eps_out, &L);
  if (rc) return rc;
  PC_REQUIRE(l > 0.0 && eps_in > 0.0 && eps_bg > 0.0 && std::isfinite(threshold), "pc_eps_gyroid: bad parameters");
  const long total = 3L * N * N * N;
  DevBuf dout;
  PC_CK(dout.reserve(sizeof(double) * total));
  eps_gyroid_kernel<<<(unsigned)((total + 255) / 256), 256>>>(N, L, l, threshold, eps_in, eps_bg, dout.as<double>());
  PC_CK_LAUNCH();
  PC_CK(cudaMemcpy(eps_out, dout.p, sizeof(double) * total, cudaMemcpyDeviceToHost));
  return PC_OK;
}

extern "C" int pc_eps_diamond(int N, const double *lattice, double l, double r, double b, double eps_in,
                              double eps_bg, double *eps_out) {
  LatMat L;
  int rc = eps_structure_common("pc_eps_diamond", N, lattice, eps_out, &L);
  if (rc) return rc;
  PC_REQUIRE(l > 0.0 && r >= 0.0 && b >= 0.0 && eps_in > 0.0 && eps_bg > 0.0, "pc_eps_diamond: bad parameters");
  const double c = 0.5 * std::sqrt(3.0) * 0.25 * l;  // half the bond length
  const double semi_major = std::sqrt(c * c + 0.25 * b * b * l * l);
  const long total = 3L * N * N * N;
  DevBuf dout;
  PC_CK(dout.reserve(sizeof(double) * total));
  eps_diamond_kernel<<<(unsigned)((total + 255) / 256), 256>>>(N, L, l, r * l, semi_major, eps_in, eps_bg,
                                                               dout.as<double>());
  PC_CK_LAUNCH();
  PC_CK(cudaMemcpy(eps_out, dout.p, sizeof(double) * total, cudaMemcpyDeviceToHost));
  return PC_OK;
}
