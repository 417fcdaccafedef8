// mf_certify.cu -- certification of traced points (Sec. V-C, App. A):
// forward kinematics of a serial DH arm and the exact distance between each
// robot element (link capsules; spheres fixed to the links, the paper's robot
// model) and each box / sphere / cylinder obstacle, in FP64; and the
// whole-cell certificate of each crossing n-simplex's manifold piece.
//
// Capsule/box distance: in the box frame the squared distance from the
// segment point p(t) = a + t (b - a) to the box is
//   F(t) = sum_i max(0, |p_i(t)| - h_i)^2,
// convex and piecewise quadratic with breakpoints where p_i(t) = +-h_i.  The
// minimum over [0,1] is found exactly by minimising the quadratic of every
// piece (at most 7).  This extends App. A's sphere/box test (a sphere is the
// zero-length capsule) to capsules.
//
// Capsule/cylinder distance: in the cylinder frame
//   F(t) = max(0, rho(t) - r_c)^2 + max(0, |z(t)| - h/2)^2,
// rho the distance to the axis, is the squared distance to the solid
// cylinder (App. A's ring-region test is its zero-length case); it is convex
// and C^1, so bracketed Newton steps on F' find its minimum and the same
// convexity certificate as for boxes proves it.
#include <cmath>
#include <vector>

#include "mf_internal.cuh"
#include "mf_ctx.h"

#define CERT_MAX_OBS 128
#define CERT_THREADS 128
#define CERT_ELEM_TIE 1e-9  // margins this close to the maximum tie
#define CERT_MAX_ELEM (MF_MAXD + MF_MAX_SPHERES)

template <typename T>
struct CertObsT {
  T R[9];
  T t[3];
  T h[3];  // box half extents; sphere radius in h[0]; cylinder radius, half height
  int type;
};
typedef CertObsT<double> CertObs;

template <typename T>
__device__ __forceinline__ T box_F(const T *a, const T *dl, const T *h, T t) {
  T s = 0;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const T p = fabs(fma(t, dl[i], a[i])) - h[i];
    if (p > (T)0) s = fma(p, p, s);
  }
  return s;
}

template <typename T>
__device__ __forceinline__ void cswap(T &x, T &y) {
  const T lo = fmin(x, y), hi = fmax(x, y);
  x = lo;
  y = hi;
}

// Squared distance from segment [a, a+dl] (box frame) to the box |p_i| <= h_i:
// the convex piecewise quadratic sum_i max(0, |a_i + t dl_i| - h_i)^2 over
// t in [0, 1] (App. A), minimised on each piece between consecutive
// breakpoints.  The breakpoints (0, 1 and the crossings of +-h_i, unused
// slots = 2) are sorted by a fixed 19-comparator network, so every array
// index is known at compile time.
template <typename T>
__device__ T seg_box_d2(const T *a, const T *dl, const T *h) {
  T bp[8];
  bp[0] = 0;
  bp[1] = 1;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    T t1 = 2, t2 = 2;
    if (dl[i] != (T)0) {
      t1 = (h[i] - a[i]) / dl[i];
      t2 = (-h[i] - a[i]) / dl[i];
      if (!(t1 > (T)0 && t1 < (T)1)) t1 = 2;
      if (!(t2 > (T)0 && t2 < (T)1)) t2 = 2;
    }
    bp[2 + 2 * i] = t1;
    bp[3 + 2 * i] = t2;
  }
  cswap(bp[0], bp[2]); cswap(bp[1], bp[3]); cswap(bp[4], bp[6]); cswap(bp[5], bp[7]);
  cswap(bp[0], bp[4]); cswap(bp[1], bp[5]); cswap(bp[2], bp[6]); cswap(bp[3], bp[7]);
  cswap(bp[0], bp[1]); cswap(bp[2], bp[3]); cswap(bp[4], bp[5]); cswap(bp[6], bp[7]);
  cswap(bp[2], bp[4]); cswap(bp[3], bp[5]);
  cswap(bp[1], bp[4]); cswap(bp[3], bp[6]);
  cswap(bp[1], bp[2]); cswap(bp[3], bp[4]); cswap(bp[5], bp[6]);
  T best = box_F<T>(a, dl, h, (T)0);
  best = fmin(best, box_F<T>(a, dl, h, (T)1));
#pragma unroll
  for (int k = 0; k < 7; k++) {
    const T ta = bp[k], tb = bp[k + 1];
    if (!(tb > ta) || tb > (T)1) continue;
    const T tm = (T)0.5 * (ta + tb);
    T A = 0, Bc = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const T p = fma(tm, dl[i], a[i]);
      T c0;
      if (p > h[i]) c0 = a[i] - h[i];
      else if (p < -h[i]) c0 = a[i] + h[i];
      else continue;
      A = fma(dl[i], dl[i], A);
      Bc = fma((T)2 * dl[i], c0, Bc);
    }
    if (A > (T)0) {
      T ts = -Bc / ((T)2 * A);
      ts = fmin(fmax(ts, ta), tb);
      best = fmin(best, box_F<T>(a, dl, h, ts));
    }
  }
  return best;
}

// Exact distance from segment [a, a+dl] (box frame) to the box in FP64, from
// a start t near the minimiser (the FP32 bound's): Newton steps on F' land on
// the minimiser of the piece they are in, and convexity certifies the result,
// min F >= F(t) - |F'(t)| (t or 1 - t).  When that leaves more than 2e-12 of
// room in the distance, the breakpoint method decides.
__device__ double seg_box_dist64(const double *a, const double *dl, const double *h, double t) {
  double F = 0.0, G = 0.0;  // F(t) and F'(t) / 2
  for (int it = 0;; it++) {
    double H = 0.0;  // F''(t) / 2
    F = 0.0;
    G = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const double p = fma(t, dl[i], a[i]);
      const double q = fabs(p) - h[i];
      if (q > 0.0) {
        F = fma(q, q, F);
        G = fma(copysign(q, p), dl[i], G);
        H = fma(dl[i], dl[i], H);
      }
    }
    if (it == 2 || !(H > 0.0)) break;
    const double tn = fmin(fmax(t - G / H, 0.0), 1.0);
    if (tn == t) break;
    t = tn;
  }
  const double D = sqrt(F);
  if (2.0 * fabs(G) * (G > 0.0 ? t : 1.0 - t) <= 2e-12 * D) return D;
  return sqrt(seg_box_d2<double>(a, dl, h));
}

// F(t), F'(t) / 2 and F''(t) / 2 of the squared segment/cylinder distance
// (cylinder frame, radius rc, half height hh).  F is convex and C^1: the
// axis term vanishes near rho = 0 and the cap term near z = 0.
template <typename T>
__device__ __forceinline__ void cyl_fgh(const T *a, const T *dl, T rc, T hh, T t, T &F, T &G, T &H) {
  const T x = fma(t, dl[0], a[0]), y = fma(t, dl[1], a[1]), z = fma(t, dl[2], a[2]);
  F = G = H = 0;
  const T rho = sqrt(fma(x, x, y * y));
  const T qr = rho - rc;
  if (qr > (T)0) {
    const T rp = fma(x, dl[0], y * dl[1]) / rho;                       // rho'
    const T rpp = (fma(dl[0], dl[0], dl[1] * dl[1]) - rp * rp) / rho;  // rho''
    F = qr * qr;
    G = qr * rp;
    H = fma(qr, rpp, rp * rp);
  }
  const T qz = fabs(z) - hh;
  if (qz > (T)0) {
    F = fma(qz, qz, F);
    G = fma(copysign(qz, z), dl[2], G);
    H = fma(dl[2], dl[2], H);
  }
}

// Exact distance from segment [a, a+dl] (cylinder frame) to the cylinder in
// FP64 from a start t: Newton steps on F' kept inside a bracket of the
// minimiser (F' is non-decreasing), until the convexity certificate
// min F >= F(t) - |F'(t)| (t or 1 - t) leaves at most 2e-12 of room in the
// distance.
__device__ double seg_cyl_dist64(const double *a, const double *dl, double rc, double hh, double t) {
  double lo = 0.0, hi = 1.0, best = INFINITY;
  for (int it = 0; it < 80; it++) {
    double F, G, H;
    cyl_fgh<double>(a, dl, rc, hh, t, F, G, H);
    best = fmin(best, F);
    const double D = sqrt(F);
    if (F == 0.0 || G == 0.0 || 2.0 * fabs(G) * (G > 0.0 ? t : 1.0 - t) <= 2e-12 * D) return D;
    if (G > 0.0) hi = t; else lo = t;
    double tn = H > 0.0 ? t - G / H : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (hi - lo <= 1e-17) break;
    t = tn;
  }
  return sqrt(best);
}

template <typename T>
__device__ __noinline__ T seg_obstacle_dist(const CertObsT<T> &o, const T *pa, const T *pb, T t0) {
  T a[3], b[3], dl[3];
  // local = R^T (p - t)
  const T wa[3] = {pa[0] - o.t[0], pa[1] - o.t[1], pa[2] - o.t[2]};
  const T wb[3] = {pb[0] - o.t[0], pb[1] - o.t[1], pb[2] - o.t[2]};
#pragma unroll
  for (int i = 0; i < 3; i++) {
    a[i] = o.R[i] * wa[0] + o.R[3 + i] * wa[1] + o.R[6 + i] * wa[2];
    b[i] = o.R[i] * wb[0] + o.R[3 + i] * wb[1] + o.R[6 + i] * wb[2];
    dl[i] = b[i] - a[i];
  }
  if (o.type == MF_BOX) return seg_box_dist64(a, dl, o.h, t0);
  if (o.type == MF_CYLINDER) return seg_cyl_dist64(a, dl, o.h[0], o.h[1], t0);
  // sphere at the local origin: clamped projection of the centre
  const T dd = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
  T t = 0;
  if (dd > (T)0) {
    t = -(a[0] * dl[0] + a[1] * dl[1] + a[2] * dl[2]) / dd;
    t = fmin(fmax(t, (T)0), (T)1);
  }
  const T c0 = fma(t, dl[0], a[0]), c1 = fma(t, dl[1], a[1]), c2 = fma(t, dl[2], a[2]);
  const T dist = sqrt(c0 * c0 + c1 * c1 + c2 * c2) - o.h[0];
  return dist > (T)0 ? dist : (T)0;
}

// Whether the local point a + t dl lies inside the obstacle shrunk by dlt
// (FP32; the point is evaluated directly, so the answer only depends on dlt
// covering the coordinates' error).
__device__ __forceinline__ bool point_deep_inside32(const CertObsT<float> &o, const float *a,
                                                    const float *dl, float t, float dlt) {
  const float x = fmaf(t, dl[0], a[0]), y = fmaf(t, dl[1], a[1]), z = fmaf(t, dl[2], a[2]);
  if (o.type == MF_BOX)
    return fabsf(x) <= o.h[0] - dlt && fabsf(y) <= o.h[1] - dlt && fabsf(z) <= o.h[2] - dlt;
  if (o.type == MF_CYLINDER) {
    const float rr = o.h[0] - dlt;
    return rr > 0.f && fmaf(x, x, y * y) <= rr * rr && fabsf(z) <= o.h[1] - dlt;
  }
  const float rr = o.h[0] - dlt;
  return rr > 0.f && fmaf(x, x, fmaf(y, y, z * z)) <= rr * rr;
}

// Lower bound on the distance from segment [pa, pb] to an obstacle, in FP32
// (eta: a bound on this routine's own rounding of the squared distance).
// Box: in the box frame F(t) = sum_i max(0, |a_i + t dl_i| - h_i)^2 is convex
// and C^1 in t; three clamped Newton steps on F' from the projection of the
// box centre reach, or come near, its minimiser t*, and convexity gives
// F(t*) >= F(t) - |F'(t)| (t or 1 - t), whatever t is.  Every lane does the
// same work (no breakpoint sort, no divergence).  Sphere: the exact distance.
// *deep: a point of the segment lies inside the obstacle shrunk by dlt (the
// distance is then exactly 0); tested only when the bound is 0.  Its
// candidates: the middle of the segment's slab-clipped interval in the
// shrunk box (boxes), the final t and the projection of the centre
// (cylinders), the closest point (spheres).  *ubd: an upper bound on the
// same distance, from the squared distance at the final t plus eta (the
// distance from one point of the segment).  Not inlined: the kernel calls
// it from three places, and one copy keeps the code in the instruction
// cache.
__device__ __noinline__ float seg_obstacle_lb32(const CertObsT<float> &o, const float *pa,
                                                const float *pb, float eta, float dlt, float *tmin,
                                                bool *deep, float *ubd) {
  const float wa[3] = {pa[0] - o.t[0], pa[1] - o.t[1], pa[2] - o.t[2]};
  const float wb[3] = {pb[0] - o.t[0], pb[1] - o.t[1], pb[2] - o.t[2]};
  float a[3], dl[3];
#pragma unroll
  for (int i = 0; i < 3; i++) {
    a[i] = o.R[i] * wa[0] + o.R[3 + i] * wa[1] + o.R[6 + i] * wa[2];
    dl[i] = (o.R[i] * wb[0] + o.R[3 + i] * wb[1] + o.R[6 + i] * wb[2]) - a[i];
  }
  const float dd = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
  float t = 0.f;
  if (dd > 0.f) t = fminf(fmaxf(-(a[0] * dl[0] + a[1] * dl[1] + a[2] * dl[2]) / dd, 0.f), 1.f);
  if (o.type == MF_CYLINDER) {
    // convex and C^1 as for boxes: three clamped Newton steps, then the
    // convexity bound
    const float tc = t;
    float F = 0.f, G = 0.f, H = 0.f;
#pragma unroll
    for (int it = 0; it <= 3; it++) {
      cyl_fgh<float>(a, dl, o.h[0], o.h[1], t, F, G, H);
      if (it < 3 && H > 0.f) t = fminf(fmaxf(t - G / H, 0.f), 1.f);
    }
    *tmin = t;
    *ubd = sqrtf(F + eta) * 1.000001f;
    const float lbF = F - 2.f * fabsf(G) * (G > 0.f ? t : 1.f - t) - eta;
    *deep = !(lbF > 0.f) &&
            (point_deep_inside32(o, a, dl, tc, dlt) || point_deep_inside32(o, a, dl, t, dlt));
    return lbF > 0.f ? sqrtf(lbF) : 0.f;
  }
  if (o.type != MF_BOX) {
    *tmin = t;
    const float c0 = fmaf(t, dl[0], a[0]), c1 = fmaf(t, dl[1], a[1]), c2 = fmaf(t, dl[2], a[2]);
    const float c2s = c0 * c0 + c1 * c1 + c2 * c2;
    const float lb = fmaxf(sqrtf(c2s) - o.h[0], 0.f);
    *ubd = fmaxf(sqrtf(c2s + eta) * 1.000001f - o.h[0], 0.f) * 1.000001f;
    *deep = !(lb > 0.f) && point_deep_inside32(o, a, dl, t, dlt);
    return lb;
  }
  float F = 0.f, G = 0.f;  // F(t) and F'(t) / 2
#pragma unroll
  for (int it = 0; it <= 3; it++) {
    float H = 0.f;  // F''(t) / 2
    F = 0.f;
    G = 0.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const float p = fmaf(t, dl[i], a[i]);
      const float q = fabsf(p) - o.h[i];
      if (q > 0.f) {
        F = fmaf(q, q, F);
        G = fmaf(copysignf(q, p), dl[i], G);
        H = fmaf(dl[i], dl[i], H);
      }
    }
    if (it < 3 && H > 0.f) t = fminf(fmaxf(t - G / H, 0.f), 1.f);
  }
  *tmin = t;
  *ubd = sqrtf(F + eta) * 1.000001f;
  const float lbF = F - 2.f * fabsf(G) * (G > 0.f ? t : 1.f - t) - eta;
  *deep = false;
  if (!(lbF > 0.f)) {
    // slab clipping against the shrunk box
    float t0 = 0.f, t1 = 1.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const float hs = o.h[i] - dlt;
      if (dl[i] != 0.f) {
        const float inv = 1.f / dl[i];
        const float ta = (-hs - a[i]) * inv, tb = (hs - a[i]) * inv;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
      }
    }
    *deep = t0 <= t1 && point_deep_inside32(o, a, dl, 0.5f * (t0 + t1), dlt);
  }
  return lbF > 0.f ? sqrtf(lbF) : 0.f;
}

// FP64 sine and cosine by table lookup (P. T. P. Tang, "Table-lookup
// algorithms for elementary functions and their error analysis", 1991):
// x = k pi/64 + r with |r| <= pi/128, pi/64 in two parts (the first has 25
// significant bits, so k P1 is exact for |k| < 2^28), sin and cos of
// j pi/64 (j = k mod 128) from the table, and sin r, cos r - 1 from their
// Taylor polynomials (the first dropped terms at |r| = pi/128: r^9/9! about
// 9e-21, i.e. 4e-19 relative, for sin r; r^10/10! about 2e-23 for cos r - 1).
#define CERT_PI64_HI 0x1.921fb5p-5
#define CERT_PI64_LO 4.966642116727561e-10
__device__ __forceinline__ void cert_sincos(double x, const double2 *tab, double *s, double *c) {
  const double kd = rint(x * 20.371832715762604);  // x 64 / pi
  if (!(fabs(kd) < 268435456.0)) {
    sincos(x, s, c);
    return;
  }
  const double r = fma(-kd, CERT_PI64_LO, fma(-kd, CERT_PI64_HI, x));
  const double2 e = tab[(int)kd & 127];  // (sin, cos)(j pi / 64)
  const double r2 = r * r;
  const double sr = fma(r * r2, fma(r2, fma(r2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), r);
  const double cm = r2 * fma(r2, fma(r2, fma(r2, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5);
  *s = fma(e.x, cm, fma(e.y, sr, e.x));
  *c = fma(e.y, cm, fma(-e.x, sr, e.y));
}

// FP32 record of a point for the whole-cell certificate: coordinates,
// margin, deciding element (int bits), padded to whole 16-byte units.
__host__ __device__ __forceinline__ int cert_rec_stride(int d) { return (d + 2 + 3) & ~3; }

// The link loops stay rolled: unrolling them per link count inlines the
// distance routines once per link and pass, which overflows the instruction
// cache (measured: 45 no-instruction stall cycles per issue).
// Elements: link capsules e < NC (NC = NL with capsules, 0 without), then
// spheres e - NC on their links.

// T <- T A with the standard DH link transform A = Rz(theta) Tz(d) Tx(a)
// Rx(alpha),
//   A = [ct, -st ca, st sa, a ct; st, ct ca, -ct sa, a st; 0, sa, ca, d],
// row by row from c0 = T[r][0:2] . (ct, st) and v = T[r][0:2] . (-st, ct)
// (30 FP64 operations instead of the 36 of the full product).
__device__ __forceinline__ void cert_dh_step(double *T, double ct, double st, double ca, double sa,
                                             double aa, double dd) {
#pragma unroll
  for (int r = 0; r < 3; r++) {
    const double t0 = T[4 * r], t1 = T[4 * r + 1], t2 = T[4 * r + 2], t3 = T[4 * r + 3];
    const double c0 = fma(t0, ct, t1 * st);
    const double v = fma(t1, ct, -(t0 * st));
    T[4 * r] = c0;
    T[4 * r + 1] = fma(v, ca, t2 * sa);
    T[4 * r + 2] = fma(t2, ca, -(v * sa));
    T[4 * r + 3] = fma(aa, c0, fma(dd, t2, t3));
  }
}

// The robot, the obstacles and the sin/cos table, per block in shared memory
// (FP32 copies, so that the FP32 passes convert nothing on the FP64 pipe).
struct CertShared {
  CertObs so[CERT_MAX_OBS];
  CertObsT<float> sof[CERT_MAX_OBS];
  double sdh[MF_MAXD * 4], srad[MF_MAXD], ssa[MF_MAXD], sca[MF_MAXD];
  float sdh32[MF_MAXD * 4], srad32[MF_MAXD], ssa32[MF_MAXD], sca32[MF_MAXD];
  double2 ssc[128];
  int ssl[MF_MAX_SPHERES];
  double ssc64[MF_MAX_SPHERES * 3], ssr64[MF_MAX_SPHERES];
  float ssc32[MF_MAX_SPHERES * 3], ssr32[MF_MAX_SPHERES];
};

__device__ __forceinline__ void cert_load_shared(CertShared &sh, int NL, const double *dh,
                                                 const double *radius, int NS,
                                                 const int32_t *sph_link, const double *sph_c,
                                                 const double *sph_r, int nobs,
                                                 const int32_t *type, const double *pose,
                                                 const double *dims, const double2 *sctab) {
  for (int i = threadIdx.x; i < 128; i += blockDim.x) sh.ssc[i] = sctab[i];
  for (int i = threadIdx.x; i < nobs; i += blockDim.x) {
    CertObs o;
    CertObsT<float> of;
    for (int k = 0; k < 9; k++) of.R[k] = (float)(o.R[k] = pose[12 * i + k]);
    for (int k = 0; k < 3; k++) of.t[k] = (float)(o.t[k] = pose[12 * i + 9 + k]);
    of.type = o.type = type[i];
    for (int k = 0; k < 3; k++) {
      double h = dims[3 * i + k];
      if (o.type == MF_BOX || (o.type == MF_CYLINDER && k == 1)) h *= 0.5;
      of.h[k] = (float)(o.h[k] = h);
    }
    sh.so[i] = o;
    sh.sof[i] = of;
  }
  for (int i = threadIdx.x; i < NL * 4; i += blockDim.x) {
    sh.sdh[i] = dh[i];
    sh.sdh32[i] = (float)dh[i];
  }
  for (int i = threadIdx.x; i < NL; i += blockDim.x) {
    sh.srad[i] = radius ? radius[i] : 0.0;
    sh.srad32[i] = (float)sh.srad[i];
    sincos(dh[4 * i + 3], &sh.ssa[i], &sh.sca[i]);
    sh.ssa32[i] = (float)sh.ssa[i];
    sh.sca32[i] = (float)sh.sca[i];
  }
  for (int i = threadIdx.x; i < NS; i += blockDim.x) {
    sh.ssl[i] = sph_link[i];
    sh.ssr64[i] = sph_r[i];
    sh.ssr32[i] = (float)sph_r[i];
    for (int k = 0; k < 3; k++) sh.ssc32[3 * i + k] = (float)(sh.ssc64[3 * i + k] = sph_c[3 * i + k]);
  }
}

// A point that at most two exact evaluations settle: its elements with a
// pair inside an obstacle (bit masks over elements 0..63, 64..) and the
// pairs (element, obstacle, FP32 start t) to evaluate (0xff: none).
struct CertRec {
  uint64_t deep_lo, deep_hi;
  float t1, t2;
  uint8_t e1, k1, e2, k2;
  int32_t loc;  // the point's thread in the block
};

// Point p: margin = max over (element, obstacle) of radius - distance, its
// verdict, deciding element and FP32 record.  FAST: after the FP32 bounds,
// a point that at most two exact pair evaluations settle returns true with
// its record in *simple for cert_simple_eval; every other point is appended
// to queue and left to a FAST = false pass.
template <bool FAST>
__device__ __noinline__ bool cert_point(const CertShared &sh, int NL, const double *radius, int NS,
                                        int nobs, const double *pts, int64_t p, int d,
                                        uint8_t *verdict, double *margin, int16_t *element,
                                        float *rec32, CertRec *simple, uint32_t *queue,
                                        unsigned long long *nq) {
  const CertObs *so = sh.so;
  const CertObsT<float> *sof = sh.sof;
  const double *sdh = sh.sdh, *srad = sh.srad, *ssa = sh.ssa, *sca = sh.sca;
  const float *sdh32 = sh.sdh32, *srad32 = sh.srad32, *ssa32 = sh.ssa32, *sca32 = sh.sca32;
  const double2 *ssc = sh.ssc;
  const int *ssl = sh.ssl;
  const double *ssc64 = sh.ssc64, *ssr64 = sh.ssr64;
  const float *ssc32 = sh.ssc32, *ssr32 = sh.ssr32;
  const int NC = radius ? NL : 0, NE = NC + NS;
  // Forward kinematics, T = T * A_i with the standard DH link transform,
  // keeping every frame origin (link i runs from origin i to origin i+1) and,
  // when the robot has spheres, every rotation.  First in FP32 for all links
  // (the lower bounds below), then in FP64 only as far along the chain as the
  // pairs that need an exact distance.
  float org32[3 * (MF_MAXD + 1)];
  float rot32[9 * (MF_MAXD + 1)];
  {
    float T[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    org32[0] = org32[1] = org32[2] = 0.f;
    for (int i = 0; i < NL; i++) {
      const float th = (float)pts[p * d + i] + sdh32[4 * i];
      const float dd = sdh32[4 * i + 1], aa = sdh32[4 * i + 2];
      float st, ct;
      sincosf(th, &st, &ct);
      const float sa = ssa32[i], ca = sca32[i];
      const float A[12] = {ct, -st * ca, st * sa, aa * ct, st, ct * ca, -ct * sa, aa * st,
                           0.f, sa, ca, dd};
      float N[12];
#pragma unroll
      for (int r = 0; r < 3; r++) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
          float v = T[4 * r + 0] * A[c] + T[4 * r + 1] * A[4 + c] + T[4 * r + 2] * A[8 + c];
          if (c == 3) v += T[4 * r + 3];
          N[4 * r + c] = v;
        }
      }
#pragma unroll
      for (int k = 0; k < 12; k++) T[k] = N[k];
      org32[3 * (i + 1) + 0] = T[3];
      org32[3 * (i + 1) + 1] = T[7];
      org32[3 * (i + 1) + 2] = T[11];
      if (NS) {
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
          for (int c = 0; c < 3; c++) rot32[9 * (i + 1) + 3 * r + c] = T[4 * r + c];
      }
    }
  }
  double T[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};  // 3x4 row-major
  double org[3 * (MF_MAXD + 1)];
  double rot[9 * (MF_MAXD + 1)];
  org[0] = org[1] = org[2] = 0.0;
  int done = 0;  // FP64 origins known: 0 .. done
  auto fk64 = [&](int upto) {
    for (int i = done; i < upto; i++) {
      double st, ct;
      cert_sincos(pts[p * d + i] + sdh[4 * i], ssc, &st, &ct);
      cert_dh_step(T, ct, st, sca[i], ssa[i], sdh[4 * i + 2], sdh[4 * i + 1]);
      org[3 * (i + 1) + 0] = T[3];
      org[3 * (i + 1) + 1] = T[7];
      org[3 * (i + 1) + 2] = T[11];
      if (NS) {
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
          for (int c = 0; c < 3; c++) rot[9 * (i + 1) + 3 * r + c] = T[4 * r + c];
      }
    }
    if (upto > done) done = upto;
  };
  // element e: its link, and its segment (a sphere is a zero-length one) in
  // FP32 from the FP32 chain
  auto elem32 = [&](int e, float *a, float *b) -> float {
    if (e < NC) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        a[c] = org32[3 * e + c];
        b[c] = org32[3 * e + 3 + c];
      }
      return srad32[e];
    }
    const int s = e - NC, f = ssl[s] + 1;
#pragma unroll
    for (int r = 0; r < 3; r++)
      a[r] = b[r] = fmaf(rot32[9 * f + 3 * r], ssc32[3 * s],
                         fmaf(rot32[9 * f + 3 * r + 1], ssc32[3 * s + 1],
                              fmaf(rot32[9 * f + 3 * r + 2], ssc32[3 * s + 2], org32[3 * f + r])));
    return ssr32[s];
  };
  // the same in FP64 (after fk64 past the element's link); one call site
  // for the chain and the distance keeps the kernel's code small
  auto exact = [&](int e, int k, double t0) -> double {
    const bool cap = e < NC;
    const int s = e - NC, f = cap ? e + 1 : ssl[s] + 1;
    fk64(f);
    double a[3], b[3], rad;
    if (cap) {
#pragma unroll
      for (int r = 0; r < 3; r++) {
        a[r] = org[3 * e + r];
        b[r] = org[3 * e + 3 + r];
      }
      rad = srad[e];
    } else {
#pragma unroll
      for (int r = 0; r < 3; r++)
        a[r] = b[r] = rot[9 * f + 3 * r] * ssc64[3 * s] + rot[9 * f + 3 * r + 1] * ssc64[3 * s + 1] +
                      rot[9 * f + 3 * r + 2] * ssc64[3 * s + 2] + org[3 * f + r];
      rad = ssr64[s];
    }
    return rad - seg_obstacle_dist(so[k], a, b, t0);
  };
  // margin = max over (element, obstacle) of radius - distance.  Every pair
  // first gets a lower bound on its distance in FP32 from the FP32 chain
  // (seg_obstacle_lb32); minus a slack of 1e-4 (1 + the largest coordinate),
  // far above the FP32 rounding of the chain (about 1e-5 of that scale), it
  // bounds the true distance from below, and radius - bound is an upper
  // bound ub on the pair's margin.  The pair with the largest ub is evaluated
  // exactly (FP64 chain to its link, FP64 distance); the others only if the
  // second-largest ub exceeds that exact margin, and then only those whose
  // ub does.  The result is the exact maximum.
  // A pair whose segment provably has a point inside the obstacle (a point
  // inside it shrunk by the same 1e-4 (1 + scale), which covers the FP32
  // chain's error in every coordinate) is at distance exactly 0: its margin
  // is the element's radius, with no FP64 work (*deep).
  auto upper = [&](int e, int k, float *tmin, bool *deep, float *lower = nullptr) -> float {
    float a[3], b[3];
    const float rad = elem32(e, a, b);
    float scale = 1.f;
#pragma unroll
    for (int c = 0; c < 3; c++)
      scale = fmaxf(scale, fmaxf(fmaxf(fabsf(a[c]), fabsf(b[c])), fabsf(sof[k].t[c]) + sof[k].h[c]));
    // local coordinates are below 2 scale: the bound's own rounding of the
    // squared distance stays far below 4e-5 (1 + scale)^2
    const float eta = 4e-5f * (1.f + scale) * (1.f + scale);
    const float sl = 1e-4f * (1.f + scale);
    float ubd;
    const float lbd = seg_obstacle_lb32(sof[k], a, b, eta, sl, tmin, deep, &ubd);
    if (lower) *lower = rad - (ubd + sl);
    return rad - (lbd - sl);
  };
  auto rad64 = [&](int e) -> double { return e < NC ? srad[e] : ssr64[e - NC]; };
  // first pass: the deep pairs fix a margin without FP64 (best_in, reached
  // first by element ein); the other pairs give bounds ub (largest ub1 at
  // (bi, bk), second ub2; per element the largest, ube, and whether it has
  // a deep pair)
  float ub1 = -INFINITY, ub2 = -INFINITY, tb = 0.f, lb1 = -INFINITY;
  // FAST: the pair with the second-largest bound (ub2) and the third bound
  float ub3 = -INFINITY, tb2 = 0.f, lb2 = -INFINITY;
  int bi2 = -1, bk2 = -1;
  int bi = -1, bk = -1, ein = -1;
  double best_in = -INFINITY;
  float ube[CERT_MAX_ELEM];
  uint64_t deep_lo = 0, deep_hi = 0;  // elements 0..63, 64..
  auto is_deep = [&](int e) -> bool {
    return e < 64 ? ((deep_lo >> e) & 1ull) != 0 : ((deep_hi >> (e - 64)) & 1ull) != 0;
  };
  for (int e = 0; e < NE; e++) {
    float um = -INFINITY;
    for (int k = 0; k < nobs; k++) {
      float tk, lbk;
      bool deep;
      const float ub = upper(e, k, &tk, &deep, &lbk);
      if (deep) {
        if (e < 64) deep_lo |= 1ull << e;
        else deep_hi |= 1ull << (e - 64);
        if (rad64(e) > best_in) {
          best_in = rad64(e);
          ein = e;
        }
        continue;
      }
      um = fmaxf(um, ub);
      if (ub > ub1) {
        if (FAST) {
          ub3 = ub2;
          bi2 = bi;
          bk2 = bk;
          tb2 = tb;
          lb2 = lb1;
        }
        ub2 = ub1;
        ub1 = ub;
        bi = e;
        bk = k;
        tb = tk;
        lb1 = lbk;
      } else if (ub > ub2) {
        if (FAST) {
          ub3 = ub2;
          bi2 = e;
          bk2 = k;
          tb2 = tk;
          lb2 = lbk;
        }
        ub2 = ub;
      } else if (FAST && ub > ub3) {
        ub3 = ub;
      }
    }
    ube[e] = um;
  }
  if (FAST) {
    // L = max(best_in, lb1, lb2) is a lower bound on the point's margin
    // (lb: the pair's margin bound from the upper distance bound of the FP32
    // chain plus the same slack).  When the third-largest bound lies below
    // L by more than the gap, only the two pairs with the largest bounds
    // (those of them whose bound reaches L - gap) can hold the maximum or tie
    // with it, besides the elements inside an obstacle (margin = radius):
    // their exact evaluations settle the point (cert_simple_eval).  The gap
    // covers the FP32 rounding of the bounds, the FP64 distance's 2e-12 and
    // the 1e-9 tie.
    const double L = fmax(best_in, (double)fmaxf(lb1, lb2));
    const double thr = L - 4e-6 * (1.0 + fabs(L));
    if (bi < 0 || (double)ub3 < thr) {
      CertRec r;
      r.deep_lo = deep_lo;
      r.deep_hi = deep_hi;
      r.e1 = r.k1 = r.e2 = r.k2 = 0xff;
      r.t1 = tb;
      r.t2 = tb2;
      r.loc = 0;
      if (bi >= 0 && (double)ub1 >= thr) {
        r.e1 = (uint8_t)bi;
        r.k1 = (uint8_t)bk;
      }
      if (bi2 >= 0 && (double)ub2 >= thr) {
        r.e2 = (uint8_t)bi2;
        r.k2 = (uint8_t)bk2;
      }
      *simple = r;
      return true;
    }
    const unsigned long long q = atomicAdd(nq, 1ull);
    queue[q] = (uint32_t)p;
    return false;
  }
  // exact margins of the other pairs: first the one with the largest bound
  // (if it can exceed best_in), then (if the second-largest bound exceeds
  // the maximum so far) every pair whose bound does
  double best = best_in;
  int be = ein;
  for (int q = -1; q < NE * nobs;) {
    int e, k;
    float t0;
    if (q < 0) {
      if (bi < 0) break;
      e = bi;
      k = bk;
      t0 = tb;
      if (!((double)ub1 > best)) break;
    } else {
      e = q / nobs;
      k = q - e * nobs;
      if (k == 0 && !((double)ube[e] > best)) {  // no pair of e can exceed best
        q += nobs;
        continue;
      }
      q++;
      if (e == bi && k == bk) continue;
      bool deep;
      if ((double)upper(e, k, &t0, &deep) <= best || deep) continue;
    }
    const double m = exact(e, k, (double)t0);
    if (m > best) {
      best = m;
      be = e;
    }
    if (q < 0) {
      if (!((double)ub2 > best)) break;
      q = 0;
    }
  }
  // the deciding element: the lowest index whose margin is within
  // CERT_ELEM_TIE of the maximum (elements inside obstacles all reach their
  // radius; the whole-cell certificate subtracts the same tolerance)
  for (int e = 0; e < be; e++) {
    // an element with a deep pair has margin exactly its radius
    bool found = is_deep(e) && rad64(e) >= best - CERT_ELEM_TIE;
    if (!is_deep(e) && (double)ube[e] >= best - CERT_ELEM_TIE) {
      for (int k = 0; k < nobs && !found; k++) {
        float t0;
        bool deep;
        if ((double)upper(e, k, &t0, &deep) >= best - CERT_ELEM_TIE)
          found = exact(e, k, (double)t0) >= best - CERT_ELEM_TIE;
      }
    }
    if (found) {
      be = e;
      break;
    }
  }
  margin[p] = best;
  verdict[p] = best >= 0.0 ? 1 : 0;
  if (element) element[p] = (int16_t)be;
  if (rec32) {  // FP32 record for the whole-cell certificate
    const int rs = cert_rec_stride(d);
    for (int k = 0; k < d; k++) rec32[p * rs + k] = (float)pts[p * d + k];
    rec32[p * rs + d] = (float)best;
    rec32[p * rs + d + 1] = __int_as_float(be);
  }
  return false;
}

// A settled point (CertRec): the FP64 chain to the deeper of the pairs'
// links, their FP64 distances from the FP32 bounds' t (the operations of
// cert_point's exact evaluation), the maximum margin with the elements
// inside an obstacle (margin = radius), the deciding element (the lowest
// index within CERT_ELEM_TIE of the maximum) and the outputs.
__device__ __forceinline__ void cert_simple_eval(const CertShared &sh, int NL, const double *radius,
                                                 const double *pts, int64_t p, int d,
                                                 const CertRec &r, uint8_t *verdict,
                                                 double *margin, int16_t *element, float *rec32) {
  const int NC = radius ? NL : 0;
  const int ec[2] = {r.e1 == 0xff ? -1 : (int)r.e1, r.e2 == 0xff ? -1 : (int)r.e2};
  const int kc[2] = {(int)r.k1, (int)r.k2};
  const double tc[2] = {(double)r.t1, (double)r.t2};
  double m[2] = {-INFINITY, -INFINITY};
  int fc[2] = {0, 0};
#pragma unroll
  for (int c = 0; c < 2; c++)
    if (ec[c] >= 0) fc[c] = ec[c] < NC ? ec[c] + 1 : sh.ssl[ec[c] - NC] + 1;
  const int fdeep = fc[0] > fc[1] ? fc[0] : fc[1];
  if (fdeep > 0) {
    double T[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    double a[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}}, b[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int i = 0; i < fdeep; i++) {
#pragma unroll
      for (int c = 0; c < 2; c++)
        if (ec[c] == i && i < NC) {
          a[c][0] = T[3];
          a[c][1] = T[7];
          a[c][2] = T[11];
        }
      double st, ct;
      cert_sincos(pts[p * d + i] + sh.sdh[4 * i], sh.ssc, &st, &ct);
      cert_dh_step(T, ct, st, sh.sca[i], sh.ssa[i], sh.sdh[4 * i + 2], sh.sdh[4 * i + 1]);
#pragma unroll
      for (int c = 0; c < 2; c++) {
        if (ec[c] < 0 || fc[c] != i + 1) continue;
        if (ec[c] < NC) {
          b[c][0] = T[3];
          b[c][1] = T[7];
          b[c][2] = T[11];
        } else {
          const int s = ec[c] - NC;
#pragma unroll
          for (int q = 0; q < 3; q++)
            a[c][q] = b[c][q] = T[4 * q] * sh.ssc64[3 * s] + T[4 * q + 1] * sh.ssc64[3 * s + 1] +
                                T[4 * q + 2] * sh.ssc64[3 * s + 2] + T[4 * q + 3];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 2; c++)
      if (ec[c] >= 0) {
        const double rad = ec[c] < NC ? sh.srad[ec[c]] : sh.ssr64[ec[c] - NC];
        m[c] = rad - seg_obstacle_dist(sh.so[kc[c]], a[c], b[c], tc[c]);
      }
  }
  auto rad64 = [&](int e) -> double { return e < NC ? sh.srad[e] : sh.ssr64[e - NC]; };
  double best = -INFINITY;
  for (uint64_t w = r.deep_lo; w; w &= w - 1) best = fmax(best, rad64(__ffsll((long long)w) - 1));
  for (uint64_t w = r.deep_hi; w; w &= w - 1)
    best = fmax(best, rad64(64 + __ffsll((long long)w) - 1));
  best = fmax(best, fmax(m[0], m[1]));
  int be = -1;
  if (best > -INFINITY) {
    const int none = 1 << 30;
    be = none;
    for (uint64_t w = r.deep_lo; w && be == none; w &= w - 1) {
      const int e = __ffsll((long long)w) - 1;
      if (rad64(e) >= best - CERT_ELEM_TIE) be = e;
    }
    for (uint64_t w = r.deep_hi; w && be == none; w &= w - 1) {
      const int e = 64 + __ffsll((long long)w) - 1;
      if (rad64(e) >= best - CERT_ELEM_TIE) be = e;
    }
#pragma unroll
    for (int c = 0; c < 2; c++)
      if (ec[c] >= 0 && ec[c] < be && m[c] >= best - CERT_ELEM_TIE) be = ec[c];
  }
  margin[p] = best;
  verdict[p] = best >= 0.0 ? 1 : 0;
  if (element) element[p] = (int16_t)be;
  if (rec32) {
    const int rs = cert_rec_stride(d);
    for (int q = 0; q < d; q++) rec32[p * rs + q] = (float)pts[p * d + q];
    rec32[p * rs + d] = (float)best;
    rec32[p * rs + d + 1] = __int_as_float(be);
  }
}

// Certification of points, first pass (thread per point): the FP32 chain and
// pair bounds of every point; the points that one exact evaluation settles
// are sorted within the block by (link depth, obstacle type) of that pair,
// so that the warps run the FP64 chain and distance with their lanes
// together, and evaluated; the others are queued for k_certify_points_rest.
#define CERT_KEYS 64
__global__ void __launch_bounds__(CERT_THREADS) k_certify_points(
    int NL, const double *dh, const double *radius, int NS, const int32_t *sph_link,
    const double *sph_c, const double *sph_r, int nobs, const int32_t *type, const double *pose,
    const double *dims, const double *pts, int64_t n, int d, const double2 *sctab, uint8_t *verdict,
    double *margin, int16_t *element, float *rec32, uint32_t *queue, unsigned long long *nq) {
  __shared__ CertShared sh;
  __shared__ int s_cnt[CERT_KEYS], s_start[CERT_KEYS];
  __shared__ CertRec s_rec[CERT_THREADS];
  __shared__ int s_n;
  cert_load_shared(sh, NL, dh, radius, NS, sph_link, sph_c, sph_r, nobs, type, pose, dims, sctab);
  for (int i = threadIdx.x; i < CERT_KEYS; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  const int64_t p0 = blockIdx.x * (int64_t)blockDim.x;
  const int64_t p = p0 + threadIdx.x;
  CertRec rec;
  bool simple = false;
  if (p < n)
    simple = cert_point<true>(sh, NL, radius, NS, nobs, pts, p, d, verdict, margin, element, rec32,
                              &rec, queue, nq);
  // counting sort of the settled points by (chain depth, obstacle type) of
  // their deeper pair within the block (key 0: no exact evaluation)
  int key = 0, pos = 0;
  if (simple) {
    const int NC = radius ? NL : 0;
    const int e1 = rec.e1 == 0xff ? -1 : rec.e1, e2 = rec.e2 == 0xff ? -1 : rec.e2;
    const int f1 = e1 < 0 ? 0 : (e1 < NC ? e1 + 1 : sh.ssl[e1 - NC] + 1);
    const int f2 = e2 < 0 ? 0 : (e2 < NC ? e2 + 1 : sh.ssl[e2 - NC] + 1);
    const int kk = f1 >= f2 ? rec.k1 : rec.k2;
    key = (f1 > f2 ? f1 : f2) * 4 + (f1 || f2 ? sh.so[kk].type + 1 : 0);
    key = key < CERT_KEYS ? key : CERT_KEYS - 1;
    pos = atomicAdd(&s_cnt[key], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive scan of the CERT_KEYS (= 64) counts: two per lane
    const int lane = threadIdx.x;
    const int c0 = s_cnt[2 * lane], c1 = s_cnt[2 * lane + 1];
    int inc = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    s_start[2 * lane] = inc - c0 - c1;
    s_start[2 * lane + 1] = inc - c1;
    if (lane == 31) s_n = inc;
  }
  __syncthreads();
  if (simple) {
    rec.loc = (int32_t)threadIdx.x;
    s_rec[s_start[key] + pos] = rec;
  }
  __syncthreads();
  if ((int)threadIdx.x < s_n) {
    const CertRec r = s_rec[threadIdx.x];
    cert_simple_eval(sh, NL, radius, pts, p0 + r.loc, d, r, verdict, margin, element, rec32);
  }
}

// Certification of points, second pass: the queued points, with the full
// search (exact evaluations of every pair whose bound can reach the maximum,
// and the deciding element's tie search).
__global__ void __launch_bounds__(CERT_THREADS) k_certify_points_rest(
    int NL, const double *dh, const double *radius, int NS, const int32_t *sph_link,
    const double *sph_c, const double *sph_r, int nobs, const int32_t *type, const double *pose,
    const double *dims, const double *pts, int d, const double2 *sctab, uint8_t *verdict,
    double *margin, int16_t *element, float *rec32, const uint32_t *queue,
    const unsigned long long *nq) {
  __shared__ CertShared sh;
  cert_load_shared(sh, NL, dh, radius, NS, sph_link, sph_c, sph_r, nobs, type, pose, dims, sctab);
  __syncthreads();
  const unsigned long long m = *nq;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x)
    cert_point<false>(sh, NL, radius, NS, nobs, pts, (int64_t)queue[i], d, verdict, margin,
                      element, rec32, nullptr, nullptr, nullptr);
}

// Whole-cell certificate (one thread per cell): with lo_k / hi_k the range of
// coordinate k over the cell's points, span_jk = max(hi_k - p_jk, p_jk - lo_k)
// and slack = max_j (margin_j - sum_k L[e_j][k] span_jk); the piece of the
// manifold in the cell (the hull of its points) is in collision when
// slack >= 0.
__global__ void k_certify_cells_whole(const int64_t *off, const int64_t *idx, int64_t n_cells,
                                      const double *pts, int d, const double *margin,
                                      const int16_t *element, const double *L, int NE,
                                      int64_t n_points, uint8_t *whole, double *slack_out,
                                      unsigned *bad) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int64_t j0 = off[c], j1 = off[c + 1];
  double lo[MF_MAXD], hi[MF_MAXD];
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  for (int64_t j = j0; j < j1; j++) {
    const int64_t i = idx[j];
    if (i < 0 || i >= n_points) {
      atomicOr(bad, 1u);
      continue;
    }
    for (int k = 0; k < d; k++) {
      const double v = pts[i * d + k];
      lo[k] = fmin(lo[k], v);
      hi[k] = fmax(hi[k], v);
    }
  }
  double slack = -INFINITY;
  for (int64_t j = j0; j < j1; j++) {
    const int64_t i = idx[j];
    if (i < 0 || i >= n_points) continue;
    const int e = element[i];
    if (e < 0 || e >= NE) continue;
    double drop = 0.0;
    for (int k = 0; k < d; k++) {
      const double v = pts[i * d + k];
      drop = fma(L[e * d + k], fmax(hi[k] - v, v - lo[k]), drop);
    }
    slack = fmax(slack, (margin[i] - CERT_ELEM_TIE) - drop);
  }
  if (whole) whole[c] = slack >= 0.0 ? 1 : 0;
  if (slack_out) slack_out[c] = slack;
}

__global__ void k_certify_cells(const int64_t *off, const int64_t *idx, int64_t n_cells,
                                const uint8_t *verdict, int64_t n_points, uint8_t *cell_verdict,
                                unsigned *bad) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  uint8_t v = 1;
  for (int64_t j = off[c]; j < off[c + 1]; j++) {
    const int64_t i = idx[j];
    if (i < 0 || i >= n_points) { atomicOr(bad, 1u); v = 0; break; }
    v &= verdict[i];
  }
  cell_verdict[c] = v;
}

// Lipschitz table L[e][k] of the robot's elements (host, FP64, from the DH
// parameters and sphere centres): the sum of the link lengths
// sqrt(d_m^2 + a_m^2) from joint k to the element's link, plus |centre| for a
// sphere; 0 for joints after the element's link.  Rounded up by 1e-12
// relative so that the device sum stays a bound.
static void lipschitz_table(int NL, const std::vector<double> &dh, bool caps, int NS,
                            const std::vector<int32_t> &sl, const std::vector<double> &sc,
                            std::vector<double> &L) {
  const int NC = caps ? NL : 0, NE = NC + NS;
  L.assign((size_t)NE * NL, 0.0);
  for (int e = 0; e < NE; e++) {
    const int link = e < NC ? e : sl[e - NC];
    double extra = 0.0;
    if (e >= NC) {
      const double *c = &sc[3 * (e - NC)];
      extra = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
    for (int k = 0; k <= link && k < NL; k++) {
      double s = extra;
      for (int m = k; m <= link; m++) s += std::hypot(dh[4 * m + 1], dh[4 * m + 2]);
      L[(size_t)e * NL + k] = s * (1.0 + 1e-12);
    }
  }
}

// The same certificate in FP32 from the points' FP32 records (coordinates
// and margin), one thread per cell.  With u = 2^-24, P the largest |p| of
// the cell and s_k the spans, the FP32 slack of point j differs from the
// exact one by at most
//   eps_j = 2 u (2 |m_j| + sum_k L_k (2 P + (d + 4) s_k))
// (rounding of the coordinates, margin and constants to FP32, of the spans,
// the products, the d-term sum and the final difference, with a factor 2 to
// spare).  The cell is decided when some point has slack_j - eps_j >= 0
// (certified) or every point has slack_j + eps_j < 0 (not certified);
// otherwise it is recomputed in FP64 from the points and margins as
// k_certify_cells_whole does.
// Rows of up to CERT_ROW_CACHE points are read once (the records stay in
// registers for the second pass); longer rows read the rest twice.
#define CERT_ROW_CACHE 9

// Range of the cell's points (lo, hi per coordinate, P = largest |p|) from
// one FP32 record (NV4 float4 units).
template <int NV4>
__device__ __forceinline__ void cert_rec_extend(const float4 (&v)[NV4], int d, float (&lo)[MF_MAXD],
                                                float (&hi)[MF_MAXD], float &P) {
#pragma unroll
  for (int q = 0; q < NV4; q++) {
    const float vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
    for (int h = 0; h < 4; h++) {
      const int k = 4 * q + h;
      if (k < MF_MAXD && k < d) {
        lo[k] = fminf(lo[k], vv[h]);
        hi[k] = fmaxf(hi[k], vv[h]);
        P = fmaxf(P, fabsf(vv[h]));
      }
    }
  }
}

// One point's FP32 slack test (see above): sets yes when it certifies the
// cell, undecided when its error bound straddles the decision.
template <int NV4>
__device__ __forceinline__ void cert_rec_test(const float4 (&v)[NV4], int d, int NE,
                                              const float (&lo)[MF_MAXD], const float (&hi)[MF_MAXD],
                                              float P, const float *L32, bool &yes, bool &undecided) {
  float m = 0.f;
  int e = -1;
#pragma unroll
  for (int q = 0; q < NV4; q++) {
    const float vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
    for (int h = 0; h < 4; h++) {
      if (4 * q + h == d) m = vv[h];
      if (4 * q + h == d + 1) e = __float_as_int(vv[h]);
    }
  }
  if (e < 0 || e >= NE) return;
  const float u = 5.9604644775390625e-08f;
  float drop = 0.f, lsum = 0.f;
#pragma unroll
  for (int q = 0; q < NV4; q++) {
    const float vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
    for (int h = 0; h < 4; h++) {
      const int k = 4 * q + h;
      if (k < MF_MAXD && k < d) {
        const float sp = fmaxf(hi[k] - vv[h], vv[h] - lo[k]);
        const float Lk = __ldg(L32 + e * d + k);
        drop = fmaf(Lk, sp, drop);
        lsum = fmaf(Lk, fmaf((float)(d + 4), sp, 2.f * P), lsum);
      }
    }
  }
  const float sl = m - drop;
  const float eps = 2.f * u * (2.f * fabsf(m) + lsum) + 1e-30f;
  // certified iff the exact slack margin - tie - drop is >= 0
  if (sl - eps >= (float)CERT_ELEM_TIE) yes = true;
  else if (sl + eps >= (float)CERT_ELEM_TIE) undecided = true;
}

template <int NV4>
__global__ void __launch_bounds__(256, 3) k_certify_cells_whole32(
    const int64_t *off, const int64_t *idx, int64_t n_cells, const float *rec32, const double *pts,
    int d, const double *margin, const int16_t *element, const float *L32, const double *L, int NE,
    int64_t n_points, uint8_t *whole, unsigned *bad, const uint8_t *verdict,
    uint8_t *cell_verdict) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int64_t j0 = off[c], j1 = off[c + 1];
  const int64_t nr = j1 - j0;
  // with cell_verdict: also the AND of the points' verdicts (k_certify_cells)
  uint32_t all = 1;
  const float4 *R4 = reinterpret_cast<const float4 *>(rec32);
  float lo[MF_MAXD], hi[MF_MAXD];
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  float P = 0.f;
  float4 cache[CERT_ROW_CACHE][NV4];
  uint32_t valid = 0;
#pragma unroll
  for (int r = 0; r < CERT_ROW_CACHE; r++) {
    const int64_t i = r < nr ? idx[j0 + r] : -1;
    const bool in = i >= 0 && i < n_points;
    if (r < nr && !in) {
      atomicOr(bad, 1u);
      all = 0;
    }
    if (cell_verdict && in) all &= verdict[i];
#pragma unroll
    for (int q = 0; q < NV4; q++)
      cache[r][q] = in ? __ldg(R4 + i * NV4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    if (in) {
      cert_rec_extend<NV4>(cache[r], d, lo, hi, P);
      valid |= 1u << r;
    }
  }
  for (int64_t j = j0 + CERT_ROW_CACHE; j < j1; j++) {
    const int64_t i = idx[j];
    if (i < 0 || i >= n_points) {
      atomicOr(bad, 1u);
      all = 0;
      continue;
    }
    if (cell_verdict) all &= verdict[i];
    float4 v[NV4];
#pragma unroll
    for (int q = 0; q < NV4; q++) v[q] = __ldg(R4 + i * NV4 + q);
    cert_rec_extend<NV4>(v, d, lo, hi, P);
  }
  if (cell_verdict) cell_verdict[c] = (uint8_t)all;
  bool yes = false, undecided = false;
#pragma unroll
  for (int r = 0; r < CERT_ROW_CACHE; r++)
    if ((valid >> r) & 1u) cert_rec_test<NV4>(cache[r], d, NE, lo, hi, P, L32, yes, undecided);
  for (int64_t j = j0 + CERT_ROW_CACHE; j < j1 && !yes; j++) {
    const int64_t i = idx[j];
    if (i < 0 || i >= n_points) continue;
    float4 v[NV4];
#pragma unroll
    for (int q = 0; q < NV4; q++) v[q] = __ldg(R4 + i * NV4 + q);
    cert_rec_test<NV4>(v, d, NE, lo, hi, P, L32, yes, undecided);
  }
  if (!yes && undecided) {
    // close to the decision: the exact FP64 certificate
    double dlo[MF_MAXD], dhi[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) {
      dlo[k] = INFINITY;
      dhi[k] = -INFINITY;
    }
    for (int64_t j = j0; j < j1; j++) {
      const int64_t i = idx[j];
      if (i < 0 || i >= n_points) continue;
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++) {
        if (k < d) {
          const double v = pts[i * d + k];
          dlo[k] = fmin(dlo[k], v);
          dhi[k] = fmax(dhi[k], v);
        }
      }
    }
    double slack = -INFINITY;
    for (int64_t j = j0; j < j1; j++) {
      const int64_t i = idx[j];
      if (i < 0 || i >= n_points) continue;
      const int e = element[i];
      if (e < 0 || e >= NE) continue;
      double drop = 0.0;
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++) {
        if (k < d) {
          const double v = pts[i * d + k];
          drop = fma(L[e * d + k], fmax(dhi[k] - v, v - dlo[k]), drop);
        }
      }
      slack = fmax(slack, (margin[i] - CERT_ELEM_TIE) - drop);
    }
    yes = slack >= 0.0;
  }
  whole[c] = yes ? 1 : 0;
}

extern "C" int mf_certify_ex(mf_ctx *ctx, const mf_robot *robot, const mf_scene *scene,
                             const double *points, int64_t n_points, int32_t d,
                             const int64_t *cell_off, const int64_t *cell_idx, int64_t n_cells,
                             const mf_certify_out *out, void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  const bool want_cells = out && (out->cell_verdict || out->cell_whole || out->cell_slack);
  if (!robot || !scene || !out || d < 1 || d > MF_MAXD || robot->n_links != d || n_points < 0 ||
      n_cells < 0 || scene->n < 0 || scene->n > CERT_MAX_OBS || !robot->dh ||
      robot->n_spheres < 0 || robot->n_spheres > MF_MAX_SPHERES ||
      (robot->n_spheres > 0 &&
       (!robot->sphere_link || !robot->sphere_center || !robot->sphere_radius)) ||
      (!robot->radius && robot->n_spheres == 0) ||
      (scene->n > 0 && (!scene->type || !scene->pose || !scene->dims)) ||
      (n_points > 0 && (!points || !out->point_verdict || !out->margin)) ||
      (n_cells > 0 && want_cells && (!cell_off || !cell_idx)) || n_points > 0xffffffffll)
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_certify: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int NL = robot->n_links, NS = robot->n_spheres;
  const int NE = (robot->radius ? NL : 0) + NS;
  const bool whole = n_cells > 0 && (out->cell_whole || out->cell_slack);
  // scratch: error word, the sin/cos table, the Lipschitz table, and the
  // per-point elements when the caller wants a whole-cell verdict only
  // (the FP32 whole-cell pass, used when the slack itself is not wanted,
  // also needs the points' FP32 records)
  const bool fast = whole && !out->cell_slack;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_tab = 256, o_L = o_tab + 128 * sizeof(double2);
  const size_t o_L32 = o_L + al((size_t)NE * NL * 8 + 8);
  const size_t o_el = o_L32 + al((size_t)NE * NL * 4 + 8);
  const size_t need_el = whole && !out->element ? al((size_t)n_points * 2 + 8) : 0;
  const size_t o_rec = o_el + need_el;
  const size_t need_rec = fast ? al((size_t)n_points * cert_rec_stride(d) * 4) : 0;
  // the queue of points left to the full search (and its length)
  const size_t o_q = o_rec + need_rec, o_nq = o_q + al((size_t)n_points * 4 + 8);
  char *scr = (char *)mf_ctx_buffer(ctx, MF_SLOT_CERT, o_nq + 256);
  if (!scr) return MF_ERR_OOM;
  unsigned *bad = (unsigned *)scr;
  const double2 *sctab = (const double2 *)(scr + o_tab);
  double *dL = (double *)(scr + o_L);
  float *dL32 = (float *)(scr + o_L32);
  float *rec32 = fast ? (float *)(scr + o_rec) : nullptr;
  int16_t *elem = out->element ? out->element : (need_el ? (int16_t *)(scr + o_el) : nullptr);
  uint32_t *queue = (uint32_t *)(scr + o_q);
  unsigned long long *nq = (unsigned long long *)(scr + o_nq);
  cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
  cudaMemsetAsync(nq, 0, sizeof(unsigned long long), st);
  {
    // (sin, cos)(j pi / 64), rounded from extended precision
    static const std::vector<double> tab = [] {
      std::vector<double> v(256);
      const long double pi = 3.141592653589793238462643383279502884L;
      for (int j = 0; j < 128; j++) {
        v[2 * j] = (double)std::sin((long double)j * pi / 64.0L);
        v[2 * j + 1] = (double)std::cos((long double)j * pi / 64.0L);
      }
      return v;
    }();
    int rc = mf_cuda_check(ctx, cudaMemcpyAsync((void *)sctab, tab.data(), 256 * sizeof(double),
                                                cudaMemcpyHostToDevice, st),
                           "mf_certify table");
    if (rc) return rc;
  }
  std::vector<double> hL;
  std::vector<float> hL32;  // kept alive until the stream synchronises
  if (whole) {
    // the table needs the DH parameters and sphere centres on the host
    std::vector<double> hdh((size_t)NL * 4), hsc((size_t)NS * 3);
    std::vector<int32_t> hsl(NS);
    int rc = mf_cuda_check(ctx, cudaMemcpyAsync(hdh.data(), robot->dh, hdh.size() * 8,
                                                cudaMemcpyDeviceToHost, st), "mf_certify dh");
    if (!rc && NS)
      rc = mf_cuda_check(ctx, cudaMemcpyAsync(hsc.data(), robot->sphere_center, hsc.size() * 8,
                                              cudaMemcpyDeviceToHost, st), "mf_certify spheres");
    if (!rc && NS)
      rc = mf_cuda_check(ctx, cudaMemcpyAsync(hsl.data(), robot->sphere_link, hsl.size() * 4,
                                              cudaMemcpyDeviceToHost, st), "mf_certify spheres");
    if (!rc) rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_certify robot");
    if (rc) return rc;
    for (int s = 0; s < NS; s++)
      if (hsl[s] < 0 || hsl[s] >= NL)
        return mf_set_error(ctx, MF_ERR_INVALID, "mf_certify: sphere %d on link %d", s, hsl[s]);
    lipschitz_table(NL, hdh, robot->radius != nullptr, NS, hsl, hsc, hL);
    hL32.resize(hL.size());
    for (size_t i = 0; i < hL.size(); i++) hL32[i] = (float)hL[i];
    if (!hL.empty()) {
      rc = mf_cuda_check(ctx, cudaMemcpyAsync(dL, hL.data(), hL.size() * 8, cudaMemcpyHostToDevice, st),
                         "mf_certify lipschitz");
      if (!rc)
        rc = mf_cuda_check(ctx, cudaMemcpyAsync(dL32, hL32.data(), hL32.size() * 4,
                                                cudaMemcpyHostToDevice, st),
                           "mf_certify lipschitz");
      if (rc) return rc;
    }
  }
  if (n_points > 0) {
    MfProfScope ps(ctx, MF_PH_CERT_PTS, st, 1, n_points);
    const unsigned g = (unsigned)((n_points + CERT_THREADS - 1) / CERT_THREADS);
    k_certify_points<<<g, CERT_THREADS, 0, st>>>(
        NL, robot->dh, robot->radius, NS, robot->sphere_link, robot->sphere_center,
        robot->sphere_radius, scene->n, scene->type, scene->pose, scene->dims, points, n_points,
        d, sctab, out->point_verdict, out->margin, elem, rec32, queue, nq);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    k_certify_points_rest<<<(unsigned)(sms > 0 ? sms * 8 : 1024), CERT_THREADS, 0, st>>>(
        NL, robot->dh, robot->radius, NS, robot->sphere_link, robot->sphere_center,
        robot->sphere_radius, scene->n, scene->type, scene->pose, scene->dims, points, d, sctab,
        out->point_verdict, out->margin, elem, rec32, queue, nq);
  }
  // the FP32 whole-cell pass also forms the cell verdicts (one read of
  // each row)
  const bool fused = fast && cert_rec_stride(d) / 4 <= 3;
  if (n_cells > 0 && out->cell_verdict && !fused) {
    MfProfScope ps(ctx, MF_PH_CERT_CELLS, st, 1, n_cells);
    k_certify_cells<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(
        cell_off, cell_idx, n_cells, out->point_verdict, n_points, out->cell_verdict, bad);
  }
  if (whole) {
    MfProfScope ps(ctx, MF_PH_CERT_CELLS, st, 1, n_cells);
    const unsigned gc = (unsigned)((n_cells + 255) / 256);
    const int nv4 = cert_rec_stride(d) / 4;
    if (fast && nv4 == 1)
      k_certify_cells_whole32<1><<<gc, 256, 0, st>>>(cell_off, cell_idx, n_cells, rec32, points, d,
                                                      out->margin, elem, dL32, dL, NE, n_points,
                                                      out->cell_whole, bad, out->point_verdict,
                                                      out->cell_verdict);
    else if (fast && nv4 == 2)
      k_certify_cells_whole32<2><<<gc, 256, 0, st>>>(cell_off, cell_idx, n_cells, rec32, points, d,
                                                      out->margin, elem, dL32, dL, NE, n_points,
                                                      out->cell_whole, bad, out->point_verdict,
                                                      out->cell_verdict);
    else if (fast)
      k_certify_cells_whole32<3><<<gc, 256, 0, st>>>(cell_off, cell_idx, n_cells, rec32, points, d,
                                                      out->margin, elem, dL32, dL, NE, n_points,
                                                      out->cell_whole, bad, out->point_verdict,
                                                      out->cell_verdict);
    else
      k_certify_cells_whole<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(
          cell_off, cell_idx, n_cells, points, d, out->margin, elem, dL, NE, n_points,
          out->cell_whole, out->cell_slack, bad);
  }
  int rc = mf_cuda_check(ctx, cudaGetLastError(), "mf_certify launch");
  if (rc) return rc;
  unsigned hb = 0;
  rc = mf_cuda_check(ctx, cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, st),
                     "mf_certify");
  if (rc) return rc;
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_certify");
  if (rc) return rc;
  mf_prof_collect(ctx);
  if (hb) return mf_set_error(ctx, MF_ERR_INVALID, "cell_edge_idx holds an index outside [0, n_points)");
  return MF_OK;
}

extern "C" int mf_certify(mf_ctx *ctx, const mf_robot *robot, const mf_scene *scene,
                          const double *points, int64_t n_points, int32_t d,
                          const int64_t *cell_off, const int64_t *cell_idx, int64_t n_cells,
                          uint8_t *point_verdict, double *margin, uint8_t *cell_verdict,
                          void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  if (n_cells > 0 && !cell_verdict)
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_certify: bad arguments");
  mf_certify_out o = {};
  o.point_verdict = point_verdict;
  o.margin = margin;
  o.cell_verdict = cell_verdict;
  return mf_certify_ex(ctx, robot, scene, points, n_points, d, cell_off, cell_idx, n_cells, &o,
                       stream);
}
