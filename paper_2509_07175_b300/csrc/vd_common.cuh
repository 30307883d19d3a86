// vd_common.cuh -- shared device definitions for libvd (sm_103a).
//
// Precision traits, warp helpers, the status / statistics words and the
// certified sign predicate used whenever an FP32 decision cannot be trusted.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vd.h"

namespace vd {

constexpr int WARP = 32;
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long EMPTY_KEY = ~0ull;
constexpr int FLAG_BOUNDARY = INT32_MIN;

// unit roundoff of each working precision
template <typename T> struct Prec;
template <> struct Prec<float> {
  using V4 = float4;
  static constexpr float U = 5.9604644775390625e-8f;  // 2^-24
  static __device__ __forceinline__ float4 mk4(float x, float y, float z, float w) { return make_float4(x, y, z, w); }
};
template <> struct Prec<double> {
  using V4 = double4;
  static constexpr double U = 1.1102230246251565e-16;  // 2^-53
  static __device__ __forceinline__ double4 mk4(double x, double y, double z, double w) {
    return make_double4(x, y, z, w);
  }
};

__device__ __forceinline__ int site_id(float4 s) { return __float_as_int(s.w); }
__device__ __forceinline__ int site_id(double4 s) { return (int)__double2loint(s.w); }
__device__ __forceinline__ float pack_id(float, int id) { return __int_as_float(id); }
__device__ __forceinline__ double pack_id(double, int id) { return __hiloint2double(0, id); }

// first error wins (status[0] = code, status[1] = source line that raised it);
// the kernel that sets it returns early, the host reads it once
__device__ __forceinline__ void set_error_at(int* status, int code, int line) {
  if (atomicCAS(status, 0, code) == 0) status[1] = line;
}
#define set_error(status, code) set_error_at((status), (code), __LINE__)

// record the first uncertain / tied float64 decision (diagnostics slots of the stats)
__device__ __forceinline__ void record_diag(unsigned long long* stats, int a, int i, int s0, int s1, int s2, int s3,
                                            int tie, int kind) {
  if (atomicCAS(stats + VD_STAT_DIAG + 7, 0ull, (unsigned long long)(kind + 1)) == 0ull) {
    stats[VD_STAT_DIAG + 0] = (unsigned long long)(long long)a;
    stats[VD_STAT_DIAG + 1] = (unsigned long long)(long long)i;
    stats[VD_STAT_DIAG + 2] = (unsigned long long)(long long)s0;
    stats[VD_STAT_DIAG + 3] = (unsigned long long)(long long)s1;
    stats[VD_STAT_DIAG + 4] = (unsigned long long)(long long)s2;
    stats[VD_STAT_DIAG + 5] = (unsigned long long)(long long)s3;
    stats[VD_STAT_DIAG + 6] = (unsigned long long)tie;
  }
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// ordered (value, index) minimum over the warp; ties go to the smaller index
template <typename T> __device__ __forceinline__ void warp_argmin(T& d, int& id) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T od = __shfl_xor_sync(FULL, d, o);
    int oi = __shfl_xor_sync(FULL, id, o);
    if (od < d || (od == d && (unsigned)oi < (unsigned)id)) { d = od; id = oi; }
  }
}
// float values >= 0 (squared distances): two warp reductions on the bit patterns
// (non-negative floats order like their bits) instead of a shuffle tree
template <> __device__ __forceinline__ void warp_argmin<float>(float& d, int& id) {
  unsigned m = __reduce_min_sync(FULL, __float_as_uint(d));
  unsigned c = __float_as_uint(d) == m ? (unsigned)id : 0xffffffffu;
  id = (int)__reduce_min_sync(FULL, c);
  d = __uint_as_float(m);
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Certified sign of c4 - n4.q for the point q where planes 0..2 meet.
//
// With N the 3x3 matrix of the first three normals and M the 4x4 matrix of the
// rows (n_r, c_r), c4 - n4.q = det M / det N.  Both determinants are evaluated
// in float64 with a running bound on their rounding error; a sign is accepted
// when the value clears its bound.  Returns +1 (inside: n4.q < c4), -1
// (outside), 0 (tie: computed value exactly zero, counted as inside by the
// caller, following the non-strict inequality of Eq. 1) and sets *certain = 0
// when the sign could not be certified.
// ---------------------------------------------------------------------------
struct ed {
  double v, e;
};
constexpr double U64 = 1.1102230246251565e-16;

__device__ __forceinline__ ed mk(double x) { return ed{x, 0.0}; }
__device__ __forceinline__ ed operator+(ed a, ed b) {
  double s = a.v + b.v;
  return ed{s, a.e + b.e + U64 * fabs(s)};
}
__device__ __forceinline__ ed operator-(ed a, ed b) {
  double s = a.v - b.v;
  return ed{s, a.e + b.e + U64 * fabs(s)};
}
__device__ __forceinline__ ed operator*(ed a, ed b) {
  double p = a.v * b.v;
  return ed{p, fabs(a.v) * b.e + fabs(b.v) * a.e + a.e * b.e + U64 * fabs(p)};
}
__device__ __forceinline__ ed neg(ed a) { return ed{-a.v, a.e}; }
__device__ __forceinline__ ed half(ed a) { return ed{0.5 * a.v, 0.5 * a.e}; }

struct ed3 {
  ed x, y, z;
};
__device__ __forceinline__ ed3 sub3(ed3 a, ed3 b) { return ed3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ ed dot3(ed3 a, ed3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ ed3 cross3(ed3 a, ed3 b) {
  return ed3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ ed3 scale3(ed3 a, double s) {  // s = +-1: exact
  return ed3{ed{a.x.v * s, a.x.e}, ed{a.y.v * s, a.y.e}, ed{a.z.v * s, a.z.e}};
}
__device__ __forceinline__ ed det3(ed3 a, ed3 b, ed3 c) { return dot3(a, cross3(b, c)); }

struct ePlane {
  ed3 n;
  ed c;
};

// Corner of three exact planes in float64 (Cramer's rule with running error
// bounds), rounded to float; w = bound on the error of the rounded coordinates
// (1e30 if the planes are not certified independent).
__device__ __forceinline__ float4 corner64(const ePlane& p0, const ePlane& p1, const ePlane& p2) {
  ed3 x12 = cross3(p1.n, p2.n), x20 = cross3(p2.n, p0.n), x01 = cross3(p0.n, p1.n);
  ed D = dot3(p0.n, x12);
  ed A[3] = {p0.c * x12.x + p1.c * x20.x + p2.c * x01.x, p0.c * x12.y + p1.c * x20.y + p2.c * x01.y,
             p0.c * x12.z + p1.c * x20.z + p2.c * x01.z};
  double den = fabs(D.v) - D.e;
  double q[3], emax = 0;
  for (int d = 0; d < 3; ++d) {
    q[d] = A[d].v / D.v;
    double e = den > 0 ? (A[d].e + fabs(q[d]) * D.e) / den + 2 * U64 * fabs(q[d]) : 1e30;
    emax = fmax(emax, e);
  }
  float qx = (float)q[0], qy = (float)q[1], qz = (float)q[2];
  double r = fmax(fabs(q[0] - (double)qx), fmax(fabs(q[1] - (double)qy), fabs(q[2] - (double)qz)));
  float e = emax < 1e29 ? (float)((emax + r) * (1 + 1e-6)) + 1e-38f : 1e30f;
  return make_float4(qx, qy, qz, e);
}

__device__ __forceinline__ int cert_sign(ed a, int* certain) {
  double b = a.e * (1.0 + 1e-12) + 1e-300;
  if (a.v > b) return 1;
  if (a.v < -b) return -1;
  *certain = 0;
  return a.v > 0 ? 1 : (a.v < 0 ? -1 : 0);
}

__device__ __forceinline__ int side_from_planes(const ePlane* p /*[4]*/, int* certain, int* tie) {
  ed dN = det3(p[0].n, p[1].n, p[2].n);
  ed dM = neg(p[0].c * det3(p[1].n, p[2].n, p[3].n)) + p[1].c * det3(p[0].n, p[2].n, p[3].n) +
          (neg(p[2].c * det3(p[0].n, p[1].n, p[3].n)) + p[3].c * dN);
  int cN = 1, cM = 1;
  int sN = cert_sign(dN, &cN);
  int sM = cert_sign(dM, &cM);
  *certain = cN && cM;
  *tie = (dM.v == 0.0);
  if (sN == 0 || sM == 0) return 0;
  return sN * sM;
}

}  // namespace vd
