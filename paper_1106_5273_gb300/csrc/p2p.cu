// Near field: the P2P kernel (Sec. 3.1, 3.6; Table 1 counts its flops) and
// the final combine / un-permute.
//
// Per pair (d = x_i - x_j, r = |d|, rho = r/sigma_j, x = rho/sqrt2, c = sqrt(2/pi)):
//   q = exp(-x^2)                       (one ex2)
//   g = 1 - q (erfcx(x) + 2x/sqrt(pi))  (Eq. 2; erfcx by a degree-3 fit in
//                                         y = 1/x = sqrt2 sigma / r, gen_cutoff_fit.py;
//                                         rho^2 < 2 uses the Taylor series of g/rho^3)
//   S = g / r^3 = 1/r^3 - q H / r^2 with H = (erfcx fit + 2x/sqrt(pi)) / r, i.e.
//       H = sqrt(2/pi)/sigma + e_0/r + e_1/r^2 + e_2/r^3 + e_3/r^4,  e_k = c_k (sqrt2 sigma)^k
//       (one Horner polynomial in 1/r: 2x/sqrt(pi) / r is the constant term)
//   T = (c q / sigma^3 - 3 S) / r^2 = S'(r)/r; the kernels carry T' = -T/3 =
//       (S - c q / (3 sigma^3)) / r^2 (no multiply by -3 per pair) and scale the
//       stretching sums by -3 once per target
//   u_i += S (gamma_j x d)                                            (Eq. 1)
//   s_i += S (gamma_j x gamma_i) + T (gamma_i . d)(gamma_j x d)       (Eq. 3)
//   or, transpose scheme (grad u)^T gamma_i:
//   s_i += S (gamma_i x gamma_j) + T (gamma_i . (gamma_j x d)) d
// The gamma_j x gamma_i part is summed as (sum_j S gamma_j) x gamma_i.  The
// self pair is skipped explicitly (its exact value is zero).  Periodic image
// pairs form the exact FP32 difference first and then add the image shift.
//
// One warp per target leaf, two target particles per lane (one when ncrit <=
// 32); the source leaves of the leaf's list are staged through shared memory
// in double-buffered chunks.  Each staged source is classified by a lower
// bound on its distance to every target of the tile (its distance to the
// targets' bounding box, rounding margin off): the singular kernel where
// g = 1 to FP32 precision (rho >= 6.5), the cutoff without the series test
// (rho^2 >= 2), or the full form; a chunk is staged grouped by class, so each
// group runs its own branch-free loop.
#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kMaxBlock = 128;
constexpr float kInv4Pi = 0.0795774715459476679f;
constexpr float kM3 = -3.f;  // T = -3 T': scales the stretching sums built from T'
// erfcx(1/y) ~ sum c_k y^k on [1/4.6, 1] (gen_cutoff_fit.py, degree 3)
constexpr float kE0 = -1.202012900e-02f, kE1 = 6.541014877e-01f, kE2 = -2.626216807e-01f,
                kE3 = 4.812366022e-02f;
// Source-leaf classes by a lower bound d_min on the pair distance:
//   kFar : d_min >= 6.5 sigma_max: 1 - g < 4e-9 and exp(-rho^2/2) < 1e-9, so
//          S = 1/r^3 and T = -3/r^5 exactly in FP32 (singular kernel);
//   kMid : d_min >= sqrt2 sigma_max: rho^2 >= 2, no series branch needed;
//   kNear: anything closer (series branch when rho^2 < 2).
constexpr int kNear = 0, kMid = 1, kFar = 2;
constexpr double kFarRho = 6.5, kMidRho = 1.4142135623730951;

constexpr double ser_coef(int k) {  // c (-1)^k / (2^k k! (2k+3))
  double d = 2.0 * k + 3.0;
  for (int i = 1; i <= k; ++i) d *= 2.0 * i;
  return ((k & 1) ? -1.0 : 1.0) * 0.79788456080286535588 / d;
}
constexpr int kSerTerms = 12;
__constant__ float cSer[kSerTerms] = {
    (float)ser_coef(0), (float)ser_coef(1), (float)ser_coef(2),  (float)ser_coef(3),
    (float)ser_coef(4), (float)ser_coef(5), (float)ser_coef(6),  (float)ser_coef(7),
    (float)ser_coef(8), (float)ser_coef(9), (float)ser_coef(10), (float)ser_coef(11)};

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Constants of one core width sigma.  The polynomial H is stored negated
// (hn = -H) so that S = 1/r^3 + q (hn / r^2) is one FMA.
struct SigK {
  float kq;   // -log2(e) / (2 sigma^2)
  float kc;   // -sqrt(2/pi) / (3 sigma^3)   (T' = (S + kc q) / r^2)
  float ku;   // 1 / sigma^2
  float is3;  // 1 / sigma^3
  float is5;  // -2 / (3 sigma^5)            (near series: T' = f'(u) is5)
  float hn0;  // -sqrt(2/pi) / sigma          (constant term of -H)
  float hn1, hn2, hn3, hn4;  // -e_0 .. -e_3,  e_k = c_k (sqrt2 sigma)^k
};

__host__ __device__ inline SigK make_sigk(float sigma) {
  SigK k;
  const double s = (double)sigma, ky = 1.4142135623730951 * s;
  k.kq = (float)(-1.4426950408889634 / (2.0 * s * s));
  k.kc = (float)(-0.79788456080286535588 / (3.0 * s * s * s));
  k.ku = (float)(1.0 / (s * s));
  k.is3 = (float)(1.0 / (s * s * s));
  k.is5 = (float)(-2.0 / (3.0 * s * s * s * s * s));
  k.hn0 = (float)(-0.79788456080286535588 / s);
  k.hn1 = (float)(-(double)kE0);
  k.hn2 = (float)(-(double)kE1 * ky);
  k.hn3 = (float)(-(double)kE2 * ky * ky);
  k.hn4 = (float)(-(double)kE3 * ky * ky * ky);
  return k;
}

// The constants of make_sigk for the mixed core width of a pair,
// sigma_ij^2 = (sigma_i^2 + sigma_j^2) / 2, in FP32 (one division and one
// rsqrt per pair).
__device__ __forceinline__ SigK sigk_mixed(float si, float sj) {
  const float s2 = 0.5f * fmaf(si, si, sj * sj);
  const float iu = 1.f / s2;        // 1 / sigma^2
  const float is = rsqrtf(s2);      // 1 / sigma
  const float sg = s2 * is;         // sigma
  const float is3 = iu * is;        // 1 / sigma^3
  SigK k;
  k.kq = -0.72134752044448170f * iu;  // -log2(e) / 2
  k.kc = -0.26596152026762179f * is3;  // -sqrt(2/pi) / 3
  k.ku = iu;
  k.is3 = is3;
  k.is5 = (-2.f / 3.f) * is3 * iu;
  k.hn0 = -0.79788456080286535588f * is;
  k.hn1 = -kE0;
  k.hn2 = -kE1 * 1.41421356237309515f * sg;
  k.hn3 = -kE2 * 2.f * s2;
  k.hn4 = -kE3 * 2.82842712474619030f * s2 * sg;
  return k;
}

// S = g/r^3 and T' = -S'(r)/(3r) for one pair (see the file header); ST = 0:
// S only (velocity without stretching).
template <int MODE, int ST = 1>
__device__ __forceinline__ void pair_ST(float r2, const SigK& K, float& S, float& T) {
  const float rinv = rsqrt_approx(r2);
  const float rinv2 = rinv * rinv;
  T = 0.f;
  if (MODE == kFar) {
    S = rinv2 * rinv;
    if (ST) T = S * rinv2;
    return;
  }
  const float rinv3 = rinv2 * rinv;
  const float q = ex2_approx(r2 * K.kq);
  // beyond the fit range (x > 4.6) exp(-x^2) < 8e-10 multiplies a bounded
  // polynomial, so g = 1 to FP32 precision without clamping
  const float hn = fmaf(fmaf(fmaf(fmaf(K.hn4, rinv, K.hn3), rinv, K.hn2), rinv, K.hn1), rinv, K.hn0);
  S = fmaf(q, rinv2 * hn, rinv3);
  if (ST) T = fmaf(K.kc, q, S) * rinv2;
  if (MODE == kNear) {
    const float u = r2 * K.ku;
    if (u < 2.f) {
      float sS = cSer[kSerTerms - 1], sT = (float)(kSerTerms - 1) * cSer[kSerTerms - 1];
#pragma unroll
      for (int k = kSerTerms - 2; k >= 0; --k) {
        sS = fmaf(sS, u, cSer[k]);
        if (ST && k >= 1) sT = fmaf(sT, u, (float)k * cSer[k]);
      }
      S = sS * K.is3;
      if (ST) T = sT * K.is5;
    }
  }
}

struct Acc {
  float ux, uy, uz, sx, sy, sz, ax, ay, az;
};

template <int MODE>
__device__ __forceinline__ void pair_acc(float dx, float dy, float dz, const float4& gj, float gix, float giy,
                                         float giz, const SigK& K, Acc& a) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float S, T;
  pair_ST<MODE>(r2, K, S, T);
  const float cx = fmaf(gj.y, dz, -gj.z * dy);
  const float cy = fmaf(gj.z, dx, -gj.x * dz);
  const float cz = fmaf(gj.x, dy, -gj.y * dx);
  a.ux = fmaf(S, cx, a.ux);
  a.uy = fmaf(S, cy, a.uy);
  a.uz = fmaf(S, cz, a.uz);
  a.ax = fmaf(S, gj.x, a.ax);
  a.ay = fmaf(S, gj.y, a.ay);
  a.az = fmaf(S, gj.z, a.az);
  const float td = T * fmaf(gix, dx, fmaf(giy, dy, giz * dz));
  a.sx = fmaf(td, cx, a.sx);
  a.sy = fmaf(td, cy, a.sy);
  a.sz = fmaf(td, cz, a.sz);
}

// Leaf-relative form used by k_p2p: with X = x - c (c the target leaf centre;
// image shifts folded into the source's X) and k_j = gamma_j x X_j staged per
// source,  sum_j S (gamma_j x d) = A x X_i - B  and
// sum_j T (gamma_i . d)(gamma_j x d) = C x X_i - D, where
// A = sum S gamma_j, B = sum S k_j, C = sum td gamma_j, D = sum td k_j, td = T' (gamma_i . d)
// (T' = -T/3, so the stretching is s = A x gamma_i - 3 (C x X_i - D)).
// Transpose scheme: with m_i = X_i x gamma_i, w = T' gamma_i . (gamma_j x d) = T' (gamma_j . m_i -
// gamma_i . k_j); C.x = sum w, D = sum w X_j, and s = gamma_i x A - 3 ((sum w) X_i - D).
struct AccR {
  float ax, ay, az, bx, by, bz, cx, cy, cz, dx, dy, dz;
};

// ST: 0 velocity only, 1 classical stretching, 2 transpose stretching.
template <int MODE, int ST>
__device__ __forceinline__ void pair_acc_rel(float dx, float dy, float dz, const float4& xj, const float4& gj,
                                             const float4& kj, float gix, float giy, float giz, float mix,
                                             float miy, float miz, const SigK& K, AccR& a) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float S, T;
  pair_ST<MODE, ST>(r2, K, S, T);
  a.ax = fmaf(S, gj.x, a.ax);
  a.ay = fmaf(S, gj.y, a.ay);
  a.az = fmaf(S, gj.z, a.az);
  a.bx = fmaf(S, kj.x, a.bx);
  a.by = fmaf(S, kj.y, a.by);
  a.bz = fmaf(S, kj.z, a.bz);
  if (ST == 0) return;
  if (ST == 2) {
    const float e = fmaf(-giz, kj.z, fmaf(-giy, kj.y, fmaf(-gix, kj.x, fmaf(gj.x, mix, fmaf(gj.y, miy, gj.z * miz)))));
    const float w = T * e;
    a.cx += w;
    a.dx = fmaf(w, xj.x, a.dx);
    a.dy = fmaf(w, xj.y, a.dy);
    a.dz = fmaf(w, xj.z, a.dz);
    return;
  }
  const float td = T * fmaf(gix, dx, fmaf(giy, dy, giz * dz));
  a.cx = fmaf(td, gj.x, a.cx);
  a.cy = fmaf(td, gj.y, a.cy);
  a.cz = fmaf(td, gj.z, a.cz);
  a.dx = fmaf(td, kj.x, a.dx);
  a.dy = fmaf(td, kj.y, a.dy);
  a.dz = fmaf(td, kj.z, a.dz);
}

template <int TPT>
struct TgtR {
  float x[TPT], y[TPT], z[TPT], gx[TPT], gy[TPT], gz[TPT];  // X_i (leaf-relative) and gamma_i
  float mx[TPT], my[TPT], mz[TPT];                          // m_i = X_i x gamma_i (transpose scheme)
  float sg[TPT];                                            // sigma_i (mixed core width)
  int self[TPT];
  AccR a[TPT];
};

// MIX (PS only): the pair's core width is sigma_ij (sigk_mixed), not sigma_j.
template <bool PS, int MODE, bool SELF, int TPT, int ST, bool MIX>
__device__ __forceinline__ void run_chunk_rel(const float4* sA, const float4* sB, const float4* sC, const SigK* sK,
                                              int jb, int je, TgtR<TPT>& t, const SigK& K0) {
#pragma unroll 4
  for (int j = jb; j < je; ++j) {
    const float4 xj = sA[j];
    const float4 gj = sB[j];
    const float4 kj = sC[j];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      if (SELF && j == t.self[q]) continue;
      pair_acc_rel<MODE, ST>(t.x[q] - xj.x, t.y[q] - xj.y, t.z[q] - xj.z, xj, gj, kj, t.gx[q], t.gy[q], t.gz[q],
                             t.mx[q], t.my[q], t.mz[q],
                             MIX ? sigk_mixed(t.sg[q], xj.w) : (PS ? sK[j] : K0), t.a[q]);
    }
  }
}

// The groups of a staged chunk: sources [0, nf) far, [nf, nf + nm) mid, the
// rest near; the self entry (not grouped) runs the near form with the self
// pair skipped.
template <bool PS, int TPT, int ST, bool MIX>
__device__ __forceinline__ void dispatch_rel(bool self, int nf, int nm, const float4* sA, const float4* sB,
                                             const float4* sC, const SigK* sK, int cnt, TgtR<TPT>& t,
                                             const SigK& K0) {
  if (self) {
    run_chunk_rel<PS, kNear, true, TPT, ST, MIX>(sA, sB, sC, sK, 0, cnt, t, K0);
    return;
  }
  if (nf > 0) run_chunk_rel<PS, kFar, false, TPT, ST, MIX>(sA, sB, sC, sK, 0, nf, t, K0);
  if (nm > 0) run_chunk_rel<PS, kMid, false, TPT, ST, MIX>(sA, sB, sC, sK, nf, nf + nm, t, K0);
  if (nf + nm < cnt) run_chunk_rel<PS, kNear, false, TPT, ST, MIX>(sA, sB, sC, sK, nf + nm, cnt, t, K0);
}

// Axis-aligned bounding box of the targets of one tile, relative to the leaf
// centre (the coordinates the targets carry).
struct TileBox {
  float lx, ly, lz, hx, hy, hz;
};

// Box of the target coordinates x[q], y[q], z[q] (q < TPT) over the warp;
// lanes flag the targets that exist (valid[q]).
template <int TPT>
__device__ __forceinline__ TileBox tile_box(const float* x, const float* y, const float* z, const bool* valid) {
  TileBox b{INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
#pragma unroll
  for (int q = 0; q < TPT; ++q)
    if (valid[q]) {
      b.lx = fminf(b.lx, x[q]);
      b.ly = fminf(b.ly, y[q]);
      b.lz = fminf(b.lz, z[q]);
      b.hx = fmaxf(b.hx, x[q]);
      b.hy = fmaxf(b.hy, y[q]);
      b.hz = fmaxf(b.hz, z[q]);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    b.lx = fminf(b.lx, __shfl_xor_sync(0xffffffffu, b.lx, o));
    b.ly = fminf(b.ly, __shfl_xor_sync(0xffffffffu, b.ly, o));
    b.lz = fminf(b.lz, __shfl_xor_sync(0xffffffffu, b.lz, o));
    b.hx = fmaxf(b.hx, __shfl_xor_sync(0xffffffffu, b.hx, o));
    b.hy = fmaxf(b.hy, __shfl_xor_sync(0xffffffffu, b.hy, o));
    b.hz = fmaxf(b.hz, __shfl_xor_sync(0xffffffffu, b.hz, o));
  }
  return b;
}

// Class of a staged source at X (relative to the target leaf centre, image
// shift included) for the targets of a tile inside box b of a leaf of radius
// Rt: the distance from X to the box bounds its distance to every target from
// below; the bound is lowered by a margin covering the FP32 rounding of the
// coordinates (which are at most d + 2 Rt in size), so the class is never
// more optimistic than exact arithmetic would give.
__device__ __forceinline__ int source_class(float X, float Y, float Z, const TileBox& b, float Rt, float smax,
                                            float margin0) {
  const float ex = fmaxf(fmaxf(b.lx - X, X - b.hx), 0.f);
  const float ey = fmaxf(fmaxf(b.ly - Y, Y - b.hy), 0.f);
  const float ez = fmaxf(fmaxf(b.lz - Z, Z - b.hz), 0.f);
  const float d = sqrtf(ex * ex + ey * ey + ez * ez);
  const float dmin = d - (margin0 + 1e-6f * (d + 2.f * Rt));
  if (dmin >= (float)kFarRho * smax) return kFar;
  if (dmin >= (float)kMidRho * smax) return kMid;
  return kNear;
}

// Staging slots of this lane's sources j = lane + 32 q (class cls[q], -1 if
// j >= cnt): far sources first, then mid, then near, each group in source
// order.  nf and nm (the far and mid counts) come out equal in every lane.
// When every source is near the slot of source j is j.
template <int TPT>
__device__ __forceinline__ void group_slots(const int* cls, int lane, int* slot, int& nf, int& nm) {
  unsigned bf[TPT], bm[TPT], bn[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    bf[q] = __ballot_sync(0xffffffffu, cls[q] == kFar);
    bm[q] = __ballot_sync(0xffffffffu, cls[q] == kMid);
    bn[q] = __ballot_sync(0xffffffffu, cls[q] == kNear);
  }
  nf = 0;
  nm = 0;
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    nf += __popc(bf[q]);
    nm += __popc(bm[q]);
  }
  const unsigned lt = (1u << lane) - 1u;
  int ef = 0, em = 0, en = 0;  // members of each class among the earlier q
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    if (cls[q] == kFar) slot[q] = ef + __popc(bf[q] & lt);
    else if (cls[q] == kMid) slot[q] = nf + em + __popc(bm[q] & lt);
    else if (cls[q] == kNear) slot[q] = nf + nm + en + __popc(bn[q] & lt);
    else slot[q] = -1;
    ef += __popc(bf[q]);
    em += __popc(bm[q]);
    en += __popc(bn[q]);
  }
}

// Pair counts by class of one warp, added to the evaluation's counters.
__device__ __forceinline__ void add_class_counts(unsigned long long* cnt, unsigned long long c_near,
                                                 unsigned long long c_mid, unsigned long long c_far) {
  if (threadIdx.x == 0) {
    if (c_near) atomicAdd(&cnt[0], c_near);
    if (c_mid) atomicAdd(&cnt[1], c_mid);
    if (c_far) atomicAdd(&cnt[2], c_far);
  }
}

// Targets held by one thread.
template <int TPT>
struct Tgt {
  float x[TPT], y[TPT], z[TPT], gx[TPT], gy[TPT], gz[TPT];
  int self[TPT];  // staged index of the target itself in the current chunk, or -1
  Acc a[TPT];
};

template <bool PS, int MODE, bool SHIFT, bool SELF, int TPT>
__device__ __forceinline__ void run_chunk(const float4* sA, const float4* sB, const SigK* sK, int cnt, Tgt<TPT>& t,
                                          float shx, float shy, float shz, const SigK& K0) {
#pragma unroll 2
  for (int j = 0; j < cnt; ++j) {
    const float4 xj = sA[j];
    const float4 gj = sB[j];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      float dx = t.x[q] - xj.x, dy = t.y[q] - xj.y, dz = t.z[q] - xj.z;
      if (SHIFT) {
        dx += shx;
        dy += shy;
        dz += shz;
      }
      if (SELF && j == t.self[q]) continue;
      pair_acc<MODE>(dx, dy, dz, gj, t.gx[q], t.gy[q], t.gz[q], PS ? sK[j] : K0, t.a[q]);
    }
  }
}



// One warp per target leaf, TPT targets per lane; source chunks of 32*TPT
// particles double-buffered (the next chunk is loaded into registers while the
// current one is computed from shared memory).  Coordinates are relative to
// the target leaf centre.
// SEG: a batch of problems; the leaf's problem supplies sigma, the class
// bounds, the image shift and the dipole correction instead of the arguments.
// ST: 0 velocity only (dg is not written), 1 classical, 2 transpose stretching.
template <bool PS, int TPT, bool SEG, int ST, bool MIX>
__global__ void __launch_bounds__(32) k_p2p(const int* __restrict__ leaves, const int2* __restrict__ off,
                                            const int2* __restrict__ list, const int* __restrict__ begin,
                                            const int* __restrict__ end, const float4* __restrict__ cf,
                                            const float4* __restrict__ A, const float4* __restrict__ B,
                                            const float* __restrict__ far_u, const float* __restrict__ far_s,
                                            const uint32_t* __restrict__ sidx, float blen, float smax, float margin0,
                                            SigK K0, const double* __restrict__ dip, const int* __restrict__ cseg,
                                            const SegP2P* __restrict__ sp, float* __restrict__ vel,
                                            float* __restrict__ dg, unsigned long long* __restrict__ ccount) {
  constexpr int CH = 32 * TPT;
  __shared__ float4 sA[2][CH], sB[2][CH], sC[2][CH];
  __shared__ SigK sK[2][PS ? CH : 1];
  const int lane = threadIdx.x;
  const int leaf = leaves[blockIdx.x];
  const int tb = begin[leaf], te = end[leaf];
  const int2 rg = off[blockIdx.x];
  const float4 lc = cf[leaf];
  float dux = dip ? (float)dip[0] : 0.f, duy = dip ? (float)dip[1] : 0.f, duz = dip ? (float)dip[2] : 0.f;
  if (SEG) {
    const SegP2P q = sp[cseg[leaf]];
    if (!PS) K0 = make_sigk(q.sigma);
    blen = q.blen;
    smax = q.smax;
    margin0 = q.margin;
    dux = q.dip[0];
    duy = q.dip[1];
    duz = q.dip[2];
  }
  float4 ra[TPT], rb[TPT];
  unsigned long long c_near = 0, c_mid = 0, c_far = 0;
  TileBox box;
  // source j of entry e, staged as X_j = (x_j - c) - shift, gamma_j, k_j = gamma_j x X_j,
  // grouped by class (the self entry in source order)
  auto stage = [&](int bb, int cnt, int img, bool self_entry, int& nf, int& nm) {
    const float shx = -(float)(img / 9 - 1) * blen, shy = -(float)((img / 3) % 3 - 1) * blen,
                shz = -(float)(img % 3 - 1) * blen;
    float X[TPT], Y[TPT], Z[TPT];
    int cls[TPT], slot[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int j = lane + 32 * q;
      X[q] = (ra[q].x - lc.x) - shx;
      Y[q] = (ra[q].y - lc.y) - shy;
      Z[q] = (ra[q].z - lc.z) - shz;
      cls[q] = j >= cnt ? -1 : self_entry ? kNear : source_class(X[q], Y[q], Z[q], box, lc.w, smax, margin0);
    }
    group_slots<TPT>(cls, lane, slot, nf, nm);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int k = slot[q];
      if (k >= 0) {
        const float4 g = rb[q];
        sA[bb][k] = make_float4(X[q], Y[q], Z[q], ra[q].w);
        sB[bb][k] = g;
        sC[bb][k] = make_float4(g.y * Z[q] - g.z * Y[q], g.z * X[q] - g.x * Z[q], g.x * Y[q] - g.y * X[q], 0.f);
        if (PS) sK[bb][k] = make_sigk(ra[q].w);
      }
    }
  };
  for (int t0 = tb; t0 < te; t0 += CH) {
    TgtR<TPT> t;
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int i = t0 + lane + 32 * q;
      float4 xi = i < te ? A[i] : lc;
      float4 gi = i < te ? B[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      t.x[q] = xi.x - lc.x;
      t.y[q] = xi.y - lc.y;
      t.z[q] = xi.z - lc.z;
      t.gx[q] = gi.x;
      t.gy[q] = gi.y;
      t.gz[q] = gi.z;
      t.sg[q] = xi.w;
      t.mx[q] = t.y[q] * gi.z - t.z[q] * gi.y;
      t.my[q] = t.z[q] * gi.x - t.x[q] * gi.z;
      t.mz[q] = t.x[q] * gi.y - t.y[q] * gi.x;
      t.a[q] = AccR{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    }
    {
      bool valid[TPT];
#pragma unroll
      for (int q = 0; q < TPT; ++q) valid[q] = t0 + lane + 32 * q < te;
      box = tile_box<TPT>(t.x, t.y, t.z, valid);
    }
    const unsigned long long nt = (unsigned long long)min(CH, te - t0);
    int cur_e = rg.x, cur_c0 = rg.x < rg.y ? begin[list[rg.x].x] : 0, cur_cnt = 0, cur_nf = 0, cur_nm = 0;
    int buf = 0;
    if (cur_e < rg.y) {
      cur_cnt = min(CH, end[list[cur_e].x] - cur_c0);
#pragma unroll
      for (int q = 0; q < TPT; ++q) {
        const int j = lane + 32 * q;
        if (j < cur_cnt) {
          ra[q] = A[cur_c0 + j];
          rb[q] = B[cur_c0 + j];
        }
      }
      const int2 e0 = list[cur_e];
      stage(0, cur_cnt, e0.y, e0.x == leaf && e0.y == kImageZero, cur_nf, cur_nm);
    }
    __syncwarp();
    while (cur_e < rg.y) {
      int ne = cur_e, nc0 = cur_c0 + CH;
      if (nc0 >= end[list[ne].x]) {
        ++ne;
        nc0 = ne < rg.y ? begin[list[ne].x] : 0;
      }
      int ncnt = 0;
      if (ne < rg.y) {
        ncnt = min(CH, end[list[ne].x] - nc0);
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
          const int j = lane + 32 * q;
          if (j < ncnt) {
            ra[q] = A[nc0 + j];
            rb[q] = B[nc0 + j];
          }
        }
      }
      const int2 ent = list[cur_e];
      const bool self = (ent.x == leaf) && ent.y == kImageZero;
#pragma unroll
      for (int q = 0; q < TPT; ++q) t.self[q] = self ? (t0 + lane + 32 * q) - cur_c0 : -1;
      dispatch_rel<PS, TPT, ST, PS && MIX>(self, cur_nf, cur_nm, sA[buf], sB[buf], sC[buf], sK[buf], cur_cnt, t,
                                           K0);
      c_far += nt * (unsigned long long)cur_nf;
      c_mid += nt * (unsigned long long)cur_nm;
      c_near += nt * (unsigned long long)(cur_cnt - cur_nf - cur_nm);
      __syncwarp();
      buf ^= 1;
      int nnf = 0, nnm = 0;
      if (ne < rg.y) {
        const int2 en = list[ne];
        stage(buf, ncnt, en.y, en.x == leaf && en.y == kImageZero, nnf, nnm);
      }
      __syncwarp();
      cur_e = ne;
      cur_c0 = nc0;
      cur_cnt = ncnt;
      cur_nf = nnf;
      cur_nm = nnm;
    }
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int i = t0 + lane + 32 * q;
      if (i >= te) continue;
      const AccR& a = t.a[q];
      const float X = t.x[q], Y = t.y[q], Z = t.z[q];
      const uint32_t o = sidx[i];
      if (vel) {  // u = A x X_i - B
        vel[3 * o] = far_u[3 * i] + kInv4Pi * ((a.ay * Z - a.az * Y) - a.bx) + dux;
        vel[3 * o + 1] = far_u[3 * i + 1] + kInv4Pi * ((a.az * X - a.ax * Z) - a.by) + duy;
        vel[3 * o + 2] = far_u[3 * i + 2] + kInv4Pi * ((a.ax * Y - a.ay * X) - a.bz) + duz;
      }
      if (ST == 1 && dg) {  // s = A x gamma_i + C x X_i - D
        const float gx = t.gx[q], gy = t.gy[q], gz = t.gz[q];
        dg[3 * o] = far_s[3 * i] + kInv4Pi * ((a.ay * gz - a.az * gy) + kM3 * ((a.cy * Z - a.cz * Y) - a.dx));
        dg[3 * o + 1] = far_s[3 * i + 1] + kInv4Pi * ((a.az * gx - a.ax * gz) + kM3 * ((a.cz * X - a.cx * Z) - a.dy));
        dg[3 * o + 2] = far_s[3 * i + 2] + kInv4Pi * ((a.ax * gy - a.ay * gx) + kM3 * ((a.cx * Y - a.cy * X) - a.dz));
      }
      if (ST == 2 && dg) {  // s = gamma_i x A + W X_i - D (W = C.x)
        const float gx = t.gx[q], gy = t.gy[q], gz = t.gz[q];
        dg[3 * o] = far_s[3 * i] + kInv4Pi * ((gy * a.az - gz * a.ay) + kM3 * (a.cx * X - a.dx));
        dg[3 * o + 1] = far_s[3 * i + 1] + kInv4Pi * ((gz * a.ax - gx * a.az) + kM3 * (a.cx * Y - a.dy));
        dg[3 * o + 2] = far_s[3 * i + 2] + kInv4Pi * ((gx * a.ay - gy * a.ax) + kM3 * (a.cx * Z - a.dz));
      }
    }
  }
  add_class_counts(ccount, c_near, c_mid, c_far);
}

// ---- Packed form: the two targets of a lane as float2 lanes of the FP32x2
// instructions (fma/mul/add .f32x2).  The FMA pipe does the same work per
// clock either way; the packed form halves the issue slots per pair, which
// is what bounds the scalar kernel.  Every element sees the same operations in
// the same order as pair_acc_rel (subtractions as additions of staged
// negated values), so each element is rounded exactly as in the scalar form.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// SigK with every constant duplicated into both lanes.
struct SigK2 {
  float2 kq, kc, ku, is3, is5, hn0, hn1, hn2, hn3, hn4;
};

__device__ __forceinline__ SigK2 make_sigk2(const SigK& K) {
  SigK2 k;
  k.kq = dup2(K.kq);
  k.kc = dup2(K.kc);
  k.ku = dup2(K.ku);
  k.is3 = dup2(K.is3);
  k.is5 = dup2(K.is5);
  k.hn0 = dup2(K.hn0);
  k.hn1 = dup2(K.hn1);
  k.hn2 = dup2(K.hn2);
  k.hn3 = dup2(K.hn3);
  k.hn4 = dup2(K.hn4);
  return k;
}

struct AccR2 {
  float2 ax, ay, az, bx, by, bz, cx, cy, cz, dx, dy, dz;
};

// S and T of two pairs (see pair_ST).
template <int MODE, int ST>
__device__ __forceinline__ void pair_ST2(float2 r2, const SigK2& K, float2& S, float2& T) {
  const float2 rinv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
  const float2 rinv2 = mul2(rinv, rinv);
  T = dup2(0.f);
  if (MODE == kFar) {
    S = mul2(rinv2, rinv);
    if (ST) T = mul2(S, rinv2);
    return;
  }
  const float2 rinv3 = mul2(rinv2, rinv);
  const float2 qa = mul2(r2, K.kq);
  const float2 q = make_float2(ex2_approx(qa.x), ex2_approx(qa.y));
  const float2 hn = fma2(fma2(fma2(fma2(K.hn4, rinv, K.hn3), rinv, K.hn2), rinv, K.hn1), rinv, K.hn0);
  S = fma2(q, mul2(rinv2, hn), rinv3);
  if (ST) T = mul2(fma2(K.kc, q, S), rinv2);
  if (MODE == kNear) {
    const float2 u = mul2(r2, K.ku);
    if (u.x < 2.f || u.y < 2.f) {
      float2 sS = dup2(cSer[kSerTerms - 1]), sT = dup2((float)(kSerTerms - 1) * cSer[kSerTerms - 1]);
#pragma unroll
      for (int k = kSerTerms - 2; k >= 0; --k) {
        sS = fma2(sS, u, dup2(cSer[k]));
        if (ST && k >= 1) sT = fma2(sT, u, dup2((float)k * cSer[k]));
      }
      const float2 Ss = mul2(sS, K.is3), Ts = mul2(sT, K.is5);
      if (u.x < 2.f) {
        S.x = Ss.x;
        T.x = Ts.x;
      }
      if (u.y < 2.f) {
        S.y = Ss.y;
        T.y = Ts.y;
      }
    }
  }
}

// Transpose scheme (ST = 2): cx accumulates W = sum w and dx, dy, dz the sum
// of w (-X_j) (the staged coordinates are negated), mx.. = m_i, ngx.. = -gamma_i.
struct TgtT2 {
  float2 mx, my, mz, ngx, ngy, ngz;
};

// One staged source (v0..v4) against the two targets of one FP32x2 chain.
// self_lo / self_hi: the staged index of each target itself (self pair
// skipped), or -1.
template <int MODE, bool SELF, int ST>
__device__ __forceinline__ void pair_x2(const float4& v0, const float4& v1, const float4& v2, const float4& v3,
                                        const float2& v4, int j, float2 tx, float2 ty, float2 tz, float2 gix,
                                        float2 giy, float2 giz, const TgtT2& tt, int self_lo, int self_hi,
                                        const SigK2& K, AccR2& a) {
  const float2 dx = add2(tx, make_float2(v0.x, v0.y));
  const float2 dy = add2(ty, make_float2(v0.z, v0.w));
  const float2 dz = add2(tz, make_float2(v1.x, v1.y));
  const float2 gjx = make_float2(v1.z, v1.w), gjy = make_float2(v2.x, v2.y), gjz = make_float2(v2.z, v2.w);
  const float2 kjx = make_float2(v3.x, v3.y), kjy = make_float2(v3.z, v3.w), kjz = v4;
  const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
  float2 S, T;
  pair_ST2<MODE, ST>(r2, K, S, T);
  float2 td = dup2(0.f);
  if (ST == 1) td = mul2(T, fma2(gix, dx, fma2(giy, dy, mul2(giz, dz))));
  if (ST == 2)
    td = mul2(T, fma2(tt.ngz, kjz, fma2(tt.ngy, kjy, fma2(tt.ngx, kjx, fma2(gjx, tt.mx, fma2(gjy, tt.my,
                                                                                          mul2(gjz, tt.mz)))))));
  if (SELF) {
    if (j == self_lo) {
      S.x = 0.f;
      td.x = 0.f;
    }
    if (j == self_hi) {
      S.y = 0.f;
      td.y = 0.f;
    }
  }
  a.ax = fma2(S, gjx, a.ax);
  a.ay = fma2(S, gjy, a.ay);
  a.az = fma2(S, gjz, a.az);
  a.bx = fma2(S, kjx, a.bx);
  a.by = fma2(S, kjy, a.by);
  a.bz = fma2(S, kjz, a.bz);
  if (ST == 0) return;
  if (ST == 2) {  // td holds w
    a.cx = add2(a.cx, td);
    a.dx = fma2(td, make_float2(v0.x, v0.y), a.dx);
    a.dy = fma2(td, make_float2(v0.z, v0.w), a.dy);
    a.dz = fma2(td, make_float2(v1.x, v1.y), a.dz);
    return;
  }
  a.cx = fma2(td, gjx, a.cx);
  a.cy = fma2(td, gjy, a.cy);
  a.cz = fma2(td, gjz, a.cz);
  a.dx = fma2(td, kjx, a.dx);
  a.dy = fma2(td, kjy, a.dy);
  a.dz = fma2(td, kjz, a.dz);
}

template <int MODE, bool SELF, int ST>
__device__ __forceinline__ void run_chunk_x2(const float4* s0, const float4* s1, const float4* s2, const float4* s3,
                                             const float2* s4, int jb, int je, float2 tx, float2 ty, float2 tz,
                                             float2 gix, float2 giy, float2 giz, const TgtT2& tt, int self_lo,
                                             int self_hi, const SigK2& K, AccR2& a) {
#pragma unroll 4
  for (int j = jb; j < je; ++j)
    pair_x2<MODE, SELF, ST>(s0[j], s1[j], s2[j], s3[j], s4[j], j, tx, ty, tz, gix, giy, giz, tt, self_lo, self_hi,
                            K, a);
}

// k_p2p for a uniform core width and two targets per lane, in the packed
// form.  Same lists, classes, staging order and output as k_p2p<false, 2, SEG>;
// the staged source holds its negated coordinates and every value twice.
template <bool SEG, int ST>
__global__ void __launch_bounds__(32) k_p2p_x2(const int* __restrict__ leaves, const int2* __restrict__ off,
                                               const int2* __restrict__ list, const int* __restrict__ begin,
                                               const int* __restrict__ end, const float4* __restrict__ cf,
                                               const float4* __restrict__ A, const float4* __restrict__ B,
                                               const float* __restrict__ far_u, const float* __restrict__ far_s,
                                               const uint32_t* __restrict__ sidx, float blen, float smax,
                                               float margin0, SigK K0, const double* __restrict__ dip,
                                               const int* __restrict__ cseg, const SegP2P* __restrict__ sp,
                                               float* __restrict__ vel, float* __restrict__ dg,
                                               unsigned long long* __restrict__ ccount) {
  constexpr int CH = 64;
  __shared__ float4 s0[2][CH], s1[2][CH], s2[2][CH], s3[2][CH];
  __shared__ float2 s4[2][CH];
  const int lane = threadIdx.x;
  const int leaf = leaves[blockIdx.x];
  const int tb = begin[leaf], te = end[leaf];
  const int2 rg = off[blockIdx.x];
  const float4 lc = cf[leaf];
  float dux = dip ? (float)dip[0] : 0.f, duy = dip ? (float)dip[1] : 0.f, duz = dip ? (float)dip[2] : 0.f;
  if (SEG) {
    const SegP2P q = sp[cseg[leaf]];
    K0 = make_sigk(q.sigma);
    blen = q.blen;
    smax = q.smax;
    margin0 = q.margin;
    dux = q.dip[0];
    duy = q.dip[1];
    duz = q.dip[2];
  }
  const SigK2 K = make_sigk2(K0);
  float4 ra[2], rb[2];
  unsigned long long c_near = 0, c_mid = 0, c_far = 0;
  TileBox box;
  auto stage = [&](int bb, int cnt, int img, bool self_entry, int& nf, int& nm) {
    const float shx = -(float)(img / 9 - 1) * blen, shy = -(float)((img / 3) % 3 - 1) * blen,
                shz = -(float)(img % 3 - 1) * blen;
    float X[2], Y[2], Z[2];
    int cls[2], slot[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      X[q] = (ra[q].x - lc.x) - shx;
      Y[q] = (ra[q].y - lc.y) - shy;
      Z[q] = (ra[q].z - lc.z) - shz;
      cls[q] = j >= cnt ? -1 : self_entry ? kNear : source_class(X[q], Y[q], Z[q], box, lc.w, smax, margin0);
    }
    group_slots<2>(cls, lane, slot, nf, nm);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int k = slot[q];
      if (k >= 0) {
        const float4 g = rb[q];
        const float kx = g.y * Z[q] - g.z * Y[q], ky = g.z * X[q] - g.x * Z[q], kz = g.x * Y[q] - g.y * X[q];
        s0[bb][k] = make_float4(-X[q], -X[q], -Y[q], -Y[q]);
        s1[bb][k] = make_float4(-Z[q], -Z[q], g.x, g.x);
        s2[bb][k] = make_float4(g.y, g.y, g.z, g.z);
        s3[bb][k] = make_float4(kx, kx, ky, ky);
        s4[bb][k] = make_float2(kz, kz);
      }
    }
  };
  for (int t0 = tb; t0 < te; t0 += CH) {
    float xs[2], ys[2], zs[2], gxs[2], gys[2], gzs[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = t0 + lane + 32 * q;
      const float4 xi = i < te ? A[i] : lc;
      const float4 gi = i < te ? B[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      xs[q] = xi.x - lc.x;
      ys[q] = xi.y - lc.y;
      zs[q] = xi.z - lc.z;
      gxs[q] = gi.x;
      gys[q] = gi.y;
      gzs[q] = gi.z;
    }
    {
      const bool valid[2] = {t0 + lane < te, t0 + lane + 32 < te};
      box = tile_box<2>(xs, ys, zs, valid);
    }
    const float2 tx = make_float2(xs[0], xs[1]), ty = make_float2(ys[0], ys[1]), tz = make_float2(zs[0], zs[1]);
    const float2 gix = make_float2(gxs[0], gxs[1]), giy = make_float2(gys[0], gys[1]),
                 giz = make_float2(gzs[0], gzs[1]);
    TgtT2 tt;
    if (ST == 2) {
      float m[3][2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        m[0][q] = ys[q] * gzs[q] - zs[q] * gys[q];
        m[1][q] = zs[q] * gxs[q] - xs[q] * gzs[q];
        m[2][q] = xs[q] * gys[q] - ys[q] * gxs[q];
      }
      tt.mx = make_float2(m[0][0], m[0][1]);
      tt.my = make_float2(m[1][0], m[1][1]);
      tt.mz = make_float2(m[2][0], m[2][1]);
      tt.ngx = make_float2(-gxs[0], -gxs[1]);
      tt.ngy = make_float2(-gys[0], -gys[1]);
      tt.ngz = make_float2(-gzs[0], -gzs[1]);
    }
    AccR2 a;
    a.ax = a.ay = a.az = a.bx = a.by = a.bz = a.cx = a.cy = a.cz = a.dx = a.dy = a.dz = dup2(0.f);
    const unsigned long long nt = (unsigned long long)min(CH, te - t0);
    int cur_e = rg.x, cur_c0 = rg.x < rg.y ? begin[list[rg.x].x] : 0, cur_cnt = 0, cur_nf = 0, cur_nm = 0;
    int buf = 0;
    if (cur_e < rg.y) {
      cur_cnt = min(CH, end[list[cur_e].x] - cur_c0);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int j = lane + 32 * q;
        if (j < cur_cnt) {
          ra[q] = A[cur_c0 + j];
          rb[q] = B[cur_c0 + j];
        }
      }
      const int2 e0 = list[cur_e];
      stage(0, cur_cnt, e0.y, e0.x == leaf && e0.y == kImageZero, cur_nf, cur_nm);
    }
    __syncwarp();
    while (cur_e < rg.y) {
      int ne = cur_e, nc0 = cur_c0 + CH;
      if (nc0 >= end[list[ne].x]) {
        ++ne;
        nc0 = ne < rg.y ? begin[list[ne].x] : 0;
      }
      int ncnt = 0;
      if (ne < rg.y) {
        ncnt = min(CH, end[list[ne].x] - nc0);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int j = lane + 32 * q;
          if (j < ncnt) {
            ra[q] = A[nc0 + j];
            rb[q] = B[nc0 + j];
          }
        }
      }
      const int2 ent = list[cur_e];
      const bool self = (ent.x == leaf) && ent.y == kImageZero;
      const float4* c0 = s0[buf];
      const float4* c1 = s1[buf];
      const float4* c2 = s2[buf];
      const float4* c3 = s3[buf];
      const float2* c4 = s4[buf];
      if (self) {
        const int slo = (t0 + lane) - cur_c0, shi = (t0 + lane + 32) - cur_c0;
        run_chunk_x2<kNear, true, ST>(c0, c1, c2, c3, c4, 0, cur_cnt, tx, ty, tz, gix, giy, giz, tt, slo, shi, K,
                                      a);
      } else {
        const int nfm = cur_nf + cur_nm;
        if (cur_nf > 0)
          run_chunk_x2<kFar, false, ST>(c0, c1, c2, c3, c4, 0, cur_nf, tx, ty, tz, gix, giy, giz, tt, -1, -1, K, a);
        if (cur_nm > 0)
          run_chunk_x2<kMid, false, ST>(c0, c1, c2, c3, c4, cur_nf, nfm, tx, ty, tz, gix, giy, giz, tt, -1, -1, K,
                                        a);
        if (nfm < cur_cnt)
          run_chunk_x2<kNear, false, ST>(c0, c1, c2, c3, c4, nfm, cur_cnt, tx, ty, tz, gix, giy, giz, tt, -1, -1,
                                         K, a);
      }
      c_far += nt * (unsigned long long)cur_nf;
      c_mid += nt * (unsigned long long)cur_nm;
      c_near += nt * (unsigned long long)(cur_cnt - cur_nf - cur_nm);
      __syncwarp();
      buf ^= 1;
      int nnf = 0, nnm = 0;
      if (ne < rg.y) {
        const int2 en = list[ne];
        stage(buf, ncnt, en.y, en.x == leaf && en.y == kImageZero, nnf, nnm);
      }
      __syncwarp();
      cur_e = ne;
      cur_c0 = nc0;
      cur_cnt = ncnt;
      cur_nf = nnf;
      cur_nm = nnm;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = t0 + lane + 32 * q;
      if (i >= te) continue;
      const float ax = q ? a.ax.y : a.ax.x, ay = q ? a.ay.y : a.ay.x, az = q ? a.az.y : a.az.x;
      const float bx = q ? a.bx.y : a.bx.x, by = q ? a.by.y : a.by.x, bz = q ? a.bz.y : a.bz.x;
      const float cx = q ? a.cx.y : a.cx.x, cy = q ? a.cy.y : a.cy.x, cz = q ? a.cz.y : a.cz.x;
      const float ex = q ? a.dx.y : a.dx.x, ey = q ? a.dy.y : a.dy.x, ez = q ? a.dz.y : a.dz.x;
      const float X = xs[q], Y = ys[q], Z = zs[q];
      const uint32_t o = sidx[i];
      if (vel) {  // u = A x X_i - B
        vel[3 * o] = far_u[3 * i] + kInv4Pi * ((ay * Z - az * Y) - bx) + dux;
        vel[3 * o + 1] = far_u[3 * i + 1] + kInv4Pi * ((az * X - ax * Z) - by) + duy;
        vel[3 * o + 2] = far_u[3 * i + 2] + kInv4Pi * ((ax * Y - ay * X) - bz) + duz;
      }
      if (ST == 2 && dg) {  // s = gamma_i x A + W X_i + (sum w (-X_j)), W = C.x
        const float gx = gxs[q], gy = gys[q], gz = gzs[q];
        dg[3 * o] = far_s[3 * i] + kInv4Pi * ((gy * az - gz * ay) + kM3 * (cx * X + ex));
        dg[3 * o + 1] = far_s[3 * i + 1] + kInv4Pi * ((gz * ax - gx * az) + kM3 * (cx * Y + ey));
        dg[3 * o + 2] = far_s[3 * i + 2] + kInv4Pi * ((gx * ay - gy * ax) + kM3 * (cx * Z + ez));
      }
      if (ST == 1 && dg) {  // s = A x gamma_i + C x X_i - D
        const float gx = gxs[q], gy = gys[q], gz = gzs[q];
        dg[3 * o] = far_s[3 * i] + kInv4Pi * ((ay * gz - az * gy) + kM3 * ((cy * Z - cz * Y) - ex));
        dg[3 * o + 1] = far_s[3 * i + 1] + kInv4Pi * ((az * gx - ax * gz) + kM3 * ((cz * X - cx * Z) - ey));
        dg[3 * o + 2] = far_s[3 * i + 2] + kInv4Pi * ((ax * gy - ay * gx) + kM3 * ((cx * Y - cy * X) - ez));
      }
    }
  }
  add_class_counts(ccount, c_near, c_mid, c_far);
}

// All pairs of one array, free space, self pair skipped (near class throughout).
template <bool PS>
__global__ void __launch_bounds__(kMaxBlock) k_direct(int64_t n, const float* __restrict__ pos,
                                                      const float* __restrict__ gam, const float* __restrict__ sig,
                                                      SigK K0, float* __restrict__ vel, float* __restrict__ dg) {
  __shared__ float4 sA[kMaxBlock], sB[kMaxBlock];
  __shared__ SigK sK[PS ? kMaxBlock : 1];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  Tgt<1> t;
  t.x[0] = t.y[0] = t.z[0] = t.gx[0] = t.gy[0] = t.gz[0] = 0.f;
  if (valid) {
    t.x[0] = pos[3 * i];
    t.y[0] = pos[3 * i + 1];
    t.z[0] = pos[3 * i + 2];
    t.gx[0] = gam[3 * i];
    t.gy[0] = gam[3 * i + 1];
    t.gz[0] = gam[3 * i + 2];
  }
  t.a[0] = Acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
    const int cnt = (int)min((int64_t)blockDim.x, n - c0);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      int64_t j = c0 + threadIdx.x;
      float s = PS ? sig[j] : 0.f;
      sA[threadIdx.x] = make_float4(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], s);
      sB[threadIdx.x] = make_float4(gam[3 * j], gam[3 * j + 1], gam[3 * j + 2], 0.f);
      if (PS) sK[threadIdx.x] = make_sigk(s);
    }
    __syncthreads();
    if (valid) {
      const bool self = i >= c0 && i < c0 + cnt;
      t.self[0] = self ? (int)(i - c0) : -1;
      if (self) run_chunk<PS, kNear, false, true, 1>(sA, sB, sK, cnt, t, 0.f, 0.f, 0.f, K0);
      else run_chunk<PS, kNear, false, false, 1>(sA, sB, sK, cnt, t, 0.f, 0.f, 0.f, K0);
    }
  }
  if (valid) {
    const Acc& a = t.a[0];
    if (vel) {
      vel[3 * i] = kInv4Pi * a.ux;
      vel[3 * i + 1] = kInv4Pi * a.uy;
      vel[3 * i + 2] = kInv4Pi * a.uz;
    }
    if (dg) {
      dg[3 * i] = kInv4Pi * (kM3 * a.sx + (a.ay * t.gz[0] - a.az * t.gy[0]));
      dg[3 * i + 1] = kInv4Pi * (kM3 * a.sy + (a.az * t.gx[0] - a.ax * t.gz[0]));
      dg[3 * i + 2] = kInv4Pi * (kM3 * a.sz + (a.ax * t.gy[0] - a.ay * t.gx[0]));
    }
  }
}

// Dipole term of the periodic lattice sum (Sec. 3.5): the cubic-order lattice
// sum exceeds the zero-mean (Ewald) field by (1/(3V)) sum_j (x_j - c0) x gamma_j;
// its negative is added to every velocity.  Two-stage fixed-order FP64 sum.
__global__ void k_dipole_partial(const float4* __restrict__ A, const float4* __restrict__ B, int64_t n,
                                 const double* __restrict__ box, double* __restrict__ part) {
  const double L = box[3];
  const double c0x = box[0] + 0.5 * L, c0y = box[1] + 0.5 * L, c0z = box[2] + 0.5 * L;
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float4 x = A[i], g = B[i];
    double X = (double)x.x - c0x, Y = (double)x.y - c0y, Z = (double)x.z - c0z;
    s[0] += Y * g.z - Z * g.y;
    s[1] += Z * g.x - X * g.z;
    s[2] += X * g.y - Y * g.x;
  }
  __shared__ double sh[3][256];
  for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_dipole_final(const double* __restrict__ part, int nb, const double* __restrict__ box,
                               double* __restrict__ dip) {
  if (threadIdx.x >= 3) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b * 3 + threadIdx.x];
  const double L = box[3];
  dip[threadIdx.x] = -s / (3.0 * L * L * L);
}

// The same correction for each problem of a batch (one CTA per problem over
// its sorted particle range), stored with the problem's near-field constants.
__global__ void __launch_bounds__(256) k_dipole_seg(const float4* __restrict__ A, const float4* __restrict__ B,
                                                    const int* __restrict__ off, const double* __restrict__ box,
                                                    SegP2P* __restrict__ sp) {
  const int sg = blockIdx.x;
  const double* bx = box + 4 * sg;
  const double L = bx[3];
  const double c0x = bx[0] + 0.5 * L, c0y = bx[1] + 0.5 * L, c0z = bx[2] + 0.5 * L;
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = off[sg] + threadIdx.x; i < off[sg + 1]; i += blockDim.x) {
    float4 x = A[i], g = B[i];
    double X = (double)x.x - c0x, Y = (double)x.y - c0y, Z = (double)x.z - c0z;
    s[0] += Y * g.z - Z * g.y;
    s[1] += Z * g.x - X * g.z;
    s[2] += X * g.y - Y * g.x;
  }
  __shared__ double sh[3][256];
  for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) sp[sg].dip[threadIdx.x] = (float)(-sh[threadIdx.x][0] / (3.0 * L * L * L));
}

}  // namespace

// The uniform dipole velocity of a periodic one-problem evaluation (the
// zero-mean convention, subtracted in the P2P epilogue).  It needs only the
// sorted particles, so it runs on the upward pass's stream beside the
// traversal, into its own partial-sum buffer.
int dipole_pass(fmm_plan p, int64_t n, cudaStream_t s) {
  if (!p->prm.periodic || p->batched || n == 0) return FMM_OK;
  const int parts = 256;
  double* scal = p->scal.as<double>();
  FMM_TRY(p->dip_part.ensure((size_t)parts * 3 * sizeof(double)));
  ++g_launches;
  k_dipole_partial<<<parts, 256, 0, s>>>(p->sortA.as<float4>(), p->sortB.as<float4>(), n, scal,
                                         p->dip_part.as<double>());
  ++g_launches;
  k_dipole_final<<<1, 32, 0, s>>>(p->dip_part.as<double>(), parts, scal, scal + kScalDipole);
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

int p2p_near(fmm_plan p, int64_t n, float sig_u, int ps, double smax, float* vel, float* dg, cudaStream_t s) {
  const double* dip = nullptr;
  double* scal = p->scal.as<double>();
  const int* cseg = p->batched ? p->c_seg.as<int>() : nullptr;
  SegP2P* sp = p->batched ? p->seg_p2p.as<SegP2P>() : nullptr;
  if (p->prm.periodic && p->batched) {
    ++g_launches;
    k_dipole_seg<<<p->nseg, 256, 0, s>>>(p->sortA.as<float4>(), p->sortB.as<float4>(), p->seg_off.as<int>(),
                                         p->seg_box.as<double>(), sp);
  } else if (p->prm.periodic) {
    dip = scal + kScalDipole;  // dipole_pass ran beside the traversal
  }
  const float blen = p->prm.periodic ? (float)p->prm.box_len : 0.f;
  SigK K0 = make_sigk(ps ? 1.f : sig_u);
  const unsigned g = (unsigned)p->nleaves;
  const int* leaves = p->leaves.as<int>();
  const int2* off = p->p2p_off.as<int2>();
  const int2* list = p->p2p_sorted.as<int2>();
  const int* cb = p->c_begin.as<int>();
  const int* ce = p->c_end.as<int>();
  const float4* cf = p->c_cf.as<float4>();
  const float4* A = p->sortA.as<float4>();
  const float4* B = p->sortB.as<float4>();
  const float* fu = p->far_u.as<float>();
  const float* fs = p->far_s.as<float>();
  const float smaxf = (float)smax;
  const float margin0 = (float)p->cf_margin;
  const bool two = p->prm.p2p_tpl ? p->prm.p2p_tpl == 2 : p->prm.ncrit > 32;
  const int mixed = ps && p->prm.sigma_rule == FMM_SIGMA_MIXED;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(scal + kScalCount + 4);
  FMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long), s));
  ++g_launches;
  // the packed kernel stages 9 KB per warp: ask for the largest shared-memory carveout
  static bool carveout_set = false;
  if (!carveout_set) {
    const void* kx2[6] = {(const void*)k_p2p_x2<false, 0>, (const void*)k_p2p_x2<false, 1>,
                          (const void*)k_p2p_x2<false, 2>, (const void*)k_p2p_x2<true, 0>,
                          (const void*)k_p2p_x2<true, 1>,  (const void*)k_p2p_x2<true, 2>};
    for (const void* k : kx2)
      FMM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    carveout_set = true;
  }
#define FMM_P2P_LAUNCH(PS_, TPT_, SEG_, ST_)                                                                      \
  do {                                                                                                            \
    if (mixed)                                                                                                    \
      k_p2p<true, TPT_, SEG_, ST_, true><<<g, 32, 0, s>>>(leaves, off, list, cb, ce, cf, A, B, fu, fs, p->sidx,    \
                                                          blen, smaxf, margin0, K0, dip, cseg, sp, vel, dg, cnt); \
    else                                                                                                          \
      k_p2p<PS_, TPT_, SEG_, ST_, false><<<g, 32, 0, s>>>(leaves, off, list, cb, ce, cf, A, B, fu, fs, p->sidx,    \
                                                          blen, smaxf, margin0, K0, dip, cseg, sp, vel, dg, cnt); \
  } while (0)
#define FMM_P2P_X2_LAUNCH(SEG_, ST_)                                                                          \
  k_p2p_x2<SEG_, ST_><<<g, 32, 0, s>>>(leaves, off, list, cb, ce, cf, A, B, fu, fs, p->sidx, blen, smaxf,     \
                                       margin0, K0, dip, cseg, sp, vel, dg, cnt)
#define FMM_P2P_ALL(ST_)                                       \
  do {                                                         \
    if (cseg) {                                                \
      if (two) {                                               \
        if (ps) FMM_P2P_LAUNCH(true, 2, true, ST_);            \
        else FMM_P2P_X2_LAUNCH(true, ST_);                     \
      } else {                                                 \
        if (ps) FMM_P2P_LAUNCH(true, 1, true, ST_);            \
        else FMM_P2P_LAUNCH(false, 1, true, ST_);              \
      }                                                        \
    } else {                                                   \
      if (two) {                                               \
        if (ps) FMM_P2P_LAUNCH(true, 2, false, ST_);           \
        else FMM_P2P_X2_LAUNCH(false, ST_);                    \
      } else {                                                 \
        if (ps) FMM_P2P_LAUNCH(true, 1, false, ST_);           \
        else FMM_P2P_LAUNCH(false, 1, false, ST_);             \
      }                                                        \
    }                                                          \
  } while (0)
  // without a stretching output the kernels skip T and the stretching sums
  if (!dg) FMM_P2P_ALL(0);
  else if (p->prm.outputs & FMM_OUT_STRETCHING_TRANSPOSE) FMM_P2P_ALL(2);
  else FMM_P2P_ALL(1);
#undef FMM_P2P_ALL
#undef FMM_P2P_LAUNCH
#undef FMM_P2P_X2_LAUNCH
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

int p2p_direct_all(int64_t n, const float* pos, const float* gam, const float* sig, float sig_u, float* vel, float* dg,
                   cudaStream_t s) {
  const int bs = 128;
  unsigned g = (unsigned)((n + bs - 1) / bs);
  SigK K0 = make_sigk(sig ? 1.f : sig_u);
  ++g_launches;
  if (sig) k_direct<true><<<g, bs, 0, s>>>(n, pos, gam, sig, K0, vel, dg);
  else k_direct<false><<<g, bs, 0, s>>>(n, pos, gam, sig, K0, vel, dg);
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

}  // namespace fmm
