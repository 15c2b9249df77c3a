// Near field: the P2P kernel (Sec. 3.1, 3.6; Table 1 counts its flops) and
// the final combine / un-permute.
//
// Per pair (d = x_i - x_j, r = |d|, rho = r/sigma_j, x = rho/sqrt2, c = sqrt(2/pi)):
//   q = exp(-x^2)                       (one ex2)
//   g = 1 - q (erfcx(x) + 2x/sqrt(pi))  (Eq. 2; erfcx by a degree-5 fit in 1/x,
//                                         gen_cutoff_fit.py; rho^2 < 2 uses the
//                                         Taylor series of g/rho^3 instead)
//   S = g / r^3,  T = (c q / sigma^3 - 3 S) / r^2 = S'(r)/r
//   u_i += S (gamma_j x d)                                            (Eq. 1)
//   s_i += S (gamma_j x gamma_i) + T (gamma_i . d)(gamma_j x d)       (Eq. 3)
// The gamma_j x gamma_i part is summed as (sum_j S gamma_j) x gamma_i.  The
// self pair is skipped explicitly (its exact value is zero).  Periodic image
// pairs form the exact FP32 difference first and then add the image shift.
//
// One CTA per target leaf, one thread per target particle; the source leaves
// of the leaf's list are staged through shared memory.
#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kMaxBlock = 128;
constexpr float kInv4Pi = 0.0795774715459476679f;
constexpr float kTwoOverSqrtPi = 1.12837916709551257f;
constexpr float kYmin = 1.0f / 4.6f;
// erfcx(1/y) ~ sum c_k y^k on [1/4.6, 1] (gen_cutoff_fit.py)
constexpr float kE0 = -6.087852495e-03f, kE1 = 6.146454486e-01f, kE2 = -1.593122702e-01f,
                kE3 = -8.516227039e-02f, kE4 = 8.483457562e-02f, kE5 = -2.133410796e-02f;

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

// Constants of one core width sigma.
struct SigK {
  float kq;   // -log2(e) / (2 sigma^2)
  float kx;   // 1 / (sqrt2 sigma)
  float ky;   // sqrt2 sigma
  float kc;   // sqrt(2/pi) / sigma^3
  float ku;   // 1 / sigma^2
  float is3;  // 1 / sigma^3
  float is5;  // 2 / sigma^5
  float pad;
};

__host__ __device__ inline SigK make_sigk(float sigma) {
  SigK k;
  double s = (double)sigma;
  k.kq = (float)(-1.4426950408889634 / (2.0 * s * s));
  k.kx = (float)(1.0 / (1.4142135623730951 * s));
  k.ky = (float)(1.4142135623730951 * s);
  k.kc = (float)(0.79788456080286535588 / (s * s * s));
  k.ku = (float)(1.0 / (s * s));
  k.is3 = (float)(1.0 / (s * s * s));
  k.is5 = (float)(2.0 / (s * s * s * s * s));
  k.pad = 0.f;
  return k;
}

__device__ __forceinline__ void pair_ST(float r2, const SigK& K, float& S, float& T) {
  const float rinv = rsqrt_approx(r2);
  const float q = ex2_approx(r2 * K.kq);
  const float r = r2 * rinv;
  const float x = r * K.kx;
  const float y = fmaxf(rinv * K.ky, kYmin);
  float F = fmaf(fmaf(fmaf(fmaf(fmaf(kE5, y, kE4), y, kE3), y, kE2), y, kE1), y, kE0);
  F = fmaf(x, kTwoOverSqrtPi, F);
  const float g = fmaf(-q, F, 1.f);
  const float rinv2 = rinv * rinv;
  S = g * rinv2 * rinv;
  T = fmaf(K.kc, q, -3.f * S) * rinv2;
  const float u = r2 * K.ku;
  if (u < 2.f) {
    float sS = cSer[kSerTerms - 1], sT = (float)(kSerTerms - 1) * cSer[kSerTerms - 1];
#pragma unroll
    for (int k = kSerTerms - 2; k >= 0; --k) {
      sS = fmaf(sS, u, cSer[k]);
      if (k >= 1) sT = fmaf(sT, u, (float)k * cSer[k]);
    }
    S = sS * K.is3;
    T = sT * K.is5;
  }
}

struct Acc {
  float ux, uy, uz, sx, sy, sz, ax, ay, az;
};

__device__ __forceinline__ void pair_acc(float dx, float dy, float dz, const float4& gj, float gix, float giy,
                                         float giz, const SigK& K, Acc& a) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float S, T;
  pair_ST(r2, K, S, T);
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

// MODE 0: plain, 1: with image shift, 2: own leaf (skip the self pair)
template <bool PS, int MODE>
__device__ __forceinline__ void source_loop(const float4* sA, const float4* sB, const SigK* sK, int cnt, float xi,
                                            float yi, float zi, float gix, float giy, float giz, float shx, float shy,
                                            float shz, int self_j, const SigK& K0, Acc& a) {
#pragma unroll 4
  for (int j = 0; j < cnt; ++j) {
    const float4 xj = sA[j];
    const float4 gj = sB[j];
    float dx = xi - xj.x, dy = yi - xj.y, dz = zi - xj.z;
    if (MODE == 1) {
      dx += shx;
      dy += shy;
      dz += shz;
    }
    if (MODE == 2 && j == self_j) continue;
    if (PS) pair_acc(dx, dy, dz, gj, gix, giy, giz, sK[j], a);
    else pair_acc(dx, dy, dz, gj, gix, giy, giz, K0, a);
  }
}

template <bool PS>
__global__ void __launch_bounds__(kMaxBlock) k_p2p(const int* __restrict__ leaves, const int2* __restrict__ off,
                                                   const int2* __restrict__ list, const int* __restrict__ begin,
                                                   const int* __restrict__ end, const float4* __restrict__ A,
                                                   const float4* __restrict__ B, const float* __restrict__ far_u,
                                                   const float* __restrict__ far_s, const uint32_t* __restrict__ sidx,
                                                   float blen, SigK K0, const double* __restrict__ dip,
                                                   float* __restrict__ vel, float* __restrict__ dg) {
  __shared__ float4 sA[kMaxBlock], sB[kMaxBlock];
  __shared__ SigK sK[PS ? kMaxBlock : 1];
  const int leaf = leaves[blockIdx.x];
  const int tb = begin[leaf], te = end[leaf];
  const int2 rg = off[blockIdx.x];
  const float dux = dip ? (float)dip[0] : 0.f, duy = dip ? (float)dip[1] : 0.f, duz = dip ? (float)dip[2] : 0.f;
  for (int t0 = tb; t0 < te; t0 += blockDim.x) {
    const int i = t0 + threadIdx.x;
    const bool valid = i < te;
    float4 xi = valid ? A[i] : make_float4(0.f, 0.f, 0.f, 1.f);
    float4 gi = valid ? B[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    Acc a = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int e = rg.x; e < rg.y; ++e) {
      const int2 ent = list[e];
      const int src = ent.x, img = ent.y;
      const int sb = begin[src], se = end[src];
      const float shx = -(float)(img / 9 - 1) * blen;
      const float shy = -(float)((img / 3) % 3 - 1) * blen;
      const float shz = -(float)(img % 3 - 1) * blen;
      const bool self = (src == leaf) && img == kImageZero;
      for (int c0 = sb; c0 < se; c0 += blockDim.x) {
        const int cnt = min((int)blockDim.x, se - c0);
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
          float4 xa = A[c0 + threadIdx.x];
          sA[threadIdx.x] = xa;
          sB[threadIdx.x] = B[c0 + threadIdx.x];
          if (PS) sK[threadIdx.x] = make_sigk(xa.w);
        }
        __syncthreads();
        if (valid) {
          if (self)
            source_loop<PS, 2>(sA, sB, sK, cnt, xi.x, xi.y, xi.z, gi.x, gi.y, gi.z, 0.f, 0.f, 0.f, i - c0, K0, a);
          else if (img != kImageZero)
            source_loop<PS, 1>(sA, sB, sK, cnt, xi.x, xi.y, xi.z, gi.x, gi.y, gi.z, shx, shy, shz, -1, K0, a);
          else
            source_loop<PS, 0>(sA, sB, sK, cnt, xi.x, xi.y, xi.z, gi.x, gi.y, gi.z, 0.f, 0.f, 0.f, -1, K0, a);
        }
      }
    }
    if (valid) {
      const uint32_t o = sidx[i];
      const float sx = a.sx + (a.ay * gi.z - a.az * gi.y);
      const float sy = a.sy + (a.az * gi.x - a.ax * gi.z);
      const float sz = a.sz + (a.ax * gi.y - a.ay * gi.x);
      if (vel) {
        vel[3 * o] = far_u[3 * i] + kInv4Pi * a.ux + dux;
        vel[3 * o + 1] = far_u[3 * i + 1] + kInv4Pi * a.uy + duy;
        vel[3 * o + 2] = far_u[3 * i + 2] + kInv4Pi * a.uz + duz;
      }
      if (dg) {
        dg[3 * o] = far_s[3 * i] + kInv4Pi * sx;
        dg[3 * o + 1] = far_s[3 * i + 1] + kInv4Pi * sy;
        dg[3 * o + 2] = far_s[3 * i + 2] + kInv4Pi * sz;
      }
    }
  }
}

// All pairs of one array, free space, self pair skipped.
template <bool PS>
__global__ void __launch_bounds__(kMaxBlock) k_direct(int64_t n, const float* __restrict__ pos,
                                                      const float* __restrict__ gam, const float* __restrict__ sig,
                                                      SigK K0, float* __restrict__ vel, float* __restrict__ dg) {
  __shared__ float4 sA[kMaxBlock], sB[kMaxBlock];
  __shared__ SigK sK[PS ? kMaxBlock : 1];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  float xi = 0.f, yi = 0.f, zi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  if (valid) {
    xi = pos[3 * i];
    yi = pos[3 * i + 1];
    zi = pos[3 * i + 2];
    gx = gam[3 * i];
    gy = gam[3 * i + 1];
    gz = gam[3 * i + 2];
  }
  Acc a = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
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
      if (i >= c0 && i < c0 + cnt)
        source_loop<PS, 2>(sA, sB, sK, cnt, xi, yi, zi, gx, gy, gz, 0.f, 0.f, 0.f, (int)(i - c0), K0, a);
      else
        source_loop<PS, 0>(sA, sB, sK, cnt, xi, yi, zi, gx, gy, gz, 0.f, 0.f, 0.f, -1, K0, a);
    }
  }
  if (valid) {
    if (vel) {
      vel[3 * i] = kInv4Pi * a.ux;
      vel[3 * i + 1] = kInv4Pi * a.uy;
      vel[3 * i + 2] = kInv4Pi * a.uz;
    }
    if (dg) {
      dg[3 * i] = kInv4Pi * (a.sx + (a.ay * gz - a.az * gy));
      dg[3 * i + 1] = kInv4Pi * (a.sy + (a.az * gx - a.ax * gz));
      dg[3 * i + 2] = kInv4Pi * (a.sz + (a.ax * gy - a.ay * gx));
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

int p2p_block(int ncrit) {
  int b = ((ncrit + 31) / 32) * 32;
  return b < 32 ? 32 : (b > kMaxBlock ? kMaxBlock : b);
}

}  // namespace

int p2p_near(fmm_plan p, int64_t n, float sig_u, int ps, float* vel, float* dg, cudaStream_t s) {
  const double* dip = nullptr;
  double* scal = p->scal.as<double>();
  if (p->prm.periodic) {
    const int parts = 256;
    FMM_TRY(p->scan_tmp.ensure((size_t)parts * 3 * sizeof(double)));
    ++g_launches;
    k_dipole_partial<<<parts, 256, 0, s>>>(p->sortA.as<float4>(), p->sortB.as<float4>(), n, scal,
                                           p->scan_tmp.as<double>());
    ++g_launches;
    k_dipole_final<<<1, 32, 0, s>>>(p->scan_tmp.as<double>(), parts, scal, scal + kScalDipole);
    dip = scal + kScalDipole;
  }
  const int bs = p2p_block(p->prm.ncrit);
  const float blen = p->prm.periodic ? (float)p->prm.box_len : 0.f;
  SigK K0 = make_sigk(ps ? 1.f : sig_u);
  ++g_launches;
  if (ps)
    k_p2p<true><<<(unsigned)p->nleaves, bs, 0, s>>>(p->leaves.as<int>(), p->p2p_off.as<int2>(),
                                                     p->p2p_sorted.as<int2>(), p->c_begin.as<int>(), p->c_end.as<int>(),
                                                     p->sortA.as<float4>(), p->sortB.as<float4>(), p->far_u.as<float>(),
                                                     p->far_s.as<float>(), p->sidx, blen, K0, dip, vel, dg);
  else
    k_p2p<false><<<(unsigned)p->nleaves, bs, 0, s>>>(p->leaves.as<int>(), p->p2p_off.as<int2>(),
                                                      p->p2p_sorted.as<int2>(), p->c_begin.as<int>(),
                                                      p->c_end.as<int>(), p->sortA.as<float4>(), p->sortB.as<float4>(),
                                                      p->far_u.as<float>(), p->far_s.as<float>(), p->sidx, blen, K0, dip,
                                                      vel, dg);
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
