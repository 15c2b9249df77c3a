// Downward pass (Sec. 3.1): L2L from the root down, then L2P at the leaves,
// giving grad and Hessian of the three vector-potential components, hence
//   u = (1/4pi) curl psi,  s = (gamma_i . grad) u          (Eqs. 1 and 3)
// for the far field, written in sorted particle order.
#include "expansions.cuh"
#include "fmm_internal.cuh"

namespace fmm {

namespace {

__global__ void __launch_bounds__(128) k_l2l(int lb, const int* __restrict__ parent, const uint64_t* __restrict__ ckey,
                                             const float* __restrict__ opT, int P, float* __restrict__ L) {
  extern __shared__ float sLp[];  // [3][P]
  const int c = lb + blockIdx.x;
  const int par = parent[c];
  const int oct = (int)(ckey[c] & 7ull);
  for (int i = threadIdx.x; i < 3 * P; i += blockDim.x) sLp[i] = L[(size_t)par * 3 * P + i];
  __syncthreads();
  const float* W = opT + (size_t)oct * P * P;
  for (int h = 0; h < 2; ++h) {
    int r = threadIdx.x + 128 * h;
    if (r >= P) break;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 8
    for (int k = 0; k < P; ++k) {
      float w = W[(size_t)k * P + r];
      a0 = fmaf(w, sLp[k], a0);
      a1 = fmaf(w, sLp[P + k], a1);
      a2 = fmaf(w, sLp[2 * P + k], a2);
    }
    L[((size_t)c * 3 + 0) * P + r] += a0;
    L[((size_t)c * 3 + 1) * P + r] += a1;
    L[((size_t)c * 3 + 2) * P + r] += a2;
  }
}

// One CTA per leaf, one thread per particle.
__global__ void __launch_bounds__(64) k_l2p(const int* __restrict__ leaves, const int* __restrict__ begin,
                                            const int* __restrict__ end, const int* __restrict__ level,
                                            const double* __restrict__ center, const double* __restrict__ box,
                                            const int* __restrict__ cseg,
                                            const float4* __restrict__ A, const float4* __restrict__ B,
                                            const float* __restrict__ L, const int4* __restrict__ tab, int p,
                                            int transpose, float* __restrict__ far_u, float* __restrict__ far_s) {
  extern __shared__ float sm[];
  const int P = p * p;
  float2* sD = reinterpret_cast<float2*>(sm);  // [3][5][P] complex, see below
  float* sL = sm + 2 * 15 * P;                 // [3][P]
  const int leaf = leaves[blockIdx.x];
  for (int i = threadIdx.x; i < 3 * P; i += blockDim.x) sL[i] = L[(size_t)leaf * 3 * P + i];
  __syncthreads();
  const int on[5] = {1, 1, 2, 2, 2};
  // The leaf's coefficients of the derivative expansions, once per leaf:
  // D[q][o][k^2+k+mm] = W_o(k, mm) L~_q(on_o + k, om_o + mm) for mm >= 0 and
  // (-1)^m W_o(k, -m) L~_q(on_o + k, om_o - m) for mm = -m < 0, so that the
  // derivative o of potential q is sum_k,m D(+m) R~_k^m + D(-m) conj(R~_k^m).
  // The table holds, per (o, k, mm), where L~ is read and the signed weights.
  for (int e = threadIdx.x; e < 5 * P; e += blockDim.x) {
    const int4 t = __ldg(tab + e);
    const float cre = __int_as_float(t.z), cim = __int_as_float(t.w);
#pragma unroll
    for (int q = 0; q < 3; ++q) sD[q * 5 * P + e] = make_float2(cre * sL[q * P + t.x], cim * sL[q * P + t.y]);
  }
  __syncthreads();
  const int b = begin[leaf], e = end[leaf];
  const double a = box[4 * (cseg ? cseg[leaf] : 0) + 3] * ldexp(1.0, -level[leaf]);
  const float inv_a = (float)(1.0 / a);
  const double cx = center[3 * leaf], cy = center[3 * leaf + 1], cz = center[3 * leaf + 2];
  for (int j = b + threadIdx.x; j < e; j += blockDim.x) {
    float4 x = A[j];
    float4 g = B[j];
    const float X = (float)((double)x.x - cx) * inv_a;
    const float Y = (float)((double)x.y - cy) * inv_a;
    const float Z = (float)((double)x.z - cz) * inv_a;
    const float r2 = X * X + Y * Y + Z * Z;
    float acc[3][5][2];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int o = 0; o < 5; ++o) acc[q][o][0] = acc[q][o][1] = 0.f;
    float dre = 1.f, dim = 0.f;  // R~_m^m
    for (int m = 0; m < p - 1; ++m) {
      if (m > 0) {
        float f = sqrtf((2.f * m - 1.f) / (2.f * m));
        float nr = f * (dre * X - dim * Y), ni = f * (dre * Y + dim * X);
        dre = nr;
        dim = ni;
      }
      float r1r = 0.f, r1i = 0.f, r0r = dre, r0i = dim;  // R~_{k-1}, R~_k
      for (int k = m; k < p - 1; ++k) {
        if (k > m) {
          float inv = rsqrtf((float)((k + m) * (k - m)));
          float aa = (2.f * k - 1.f) * Z;
          float vr = aa * r0r, vi = aa * r0i;
          if (k - 2 >= m) {
            float bb = r2 * sqrtf((float)((k + m - 1) * (k - m - 1)));
            vr -= bb * r1r;
            vi -= bb * r1i;
          }
          r1r = r0r;
          r1i = r0i;
          r0r = vr * inv;
          r0i = vi * inv;
        }
        // contributions of R~_k^{+m} and R~_k^{-m}
#pragma unroll
        for (int o = 0; o < 5; ++o) {
          if (on[o] + k > p - 1) continue;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float2 d = sD[(q * 5 + o) * P + k * k + k + m];
            acc[q][o][0] = fmaf(d.x, r0r, fmaf(-d.y, r0i, acc[q][o][0]));
            acc[q][o][1] = fmaf(d.x, r0i, fmaf(d.y, r0r, acc[q][o][1]));
          }
          if (m > 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {  // conj(R~_k^m)
              const float2 d = sD[(q * 5 + o) * P + k * k + k - m];
              acc[q][o][0] = fmaf(d.x, r0r, fmaf(d.y, r0i, acc[q][o][0]));
              acc[q][o][1] = fmaf(-d.x, r0i, fmaf(d.y, r0r, acc[q][o][1]));
            }
          }
        }
      }
    }
    // grad / Hessian of Phi_q (unnormalized: L'_n' = a^-(n'+1) acc)
    const float s2 = inv_a * inv_a, s3 = s2 * inv_a;
    float G[3][3], H[3][3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      G[q][0] = acc[q][1][0] * s2;
      G[q][1] = -acc[q][1][1] * s2;
      G[q][2] = acc[q][0][0] * s2;
      float L0 = acc[q][2][0] * s3, a1 = acc[q][3][0] * s3, b1 = acc[q][3][1] * s3;
      float a2 = acc[q][4][0] * s3, b2 = acc[q][4][1] * s3;
      H[q][0][0] = 0.5f * (a2 - L0);
      H[q][1][1] = 0.5f * (-a2 - L0);
      H[q][2][2] = L0;
      H[q][0][1] = H[q][1][0] = -0.5f * b2;
      H[q][0][2] = H[q][2][0] = a1;
      H[q][1][2] = H[q][2][1] = -b1;
    }
    const float c4 = 0.0795774715459476679f;
    float ux = G[2][1] - G[1][2], uy = G[0][2] - G[2][0], uz = G[1][0] - G[0][1];
    const float gv[3] = {g.x, g.y, g.z};
    float sx = 0.f, sy = 0.f, sz = 0.f;
    if (transpose) {  // s_d = sum_l gamma_l d u_l / d x_d
      float sd[3];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        sd[d] = gv[0] * (H[2][d][1] - H[1][d][2]) + gv[1] * (H[0][d][2] - H[2][d][0]) +
                gv[2] * (H[1][d][0] - H[0][d][1]);
      sx = sd[0];
      sy = sd[1];
      sz = sd[2];
    } else {  // s_l = sum_d gamma_d d u_l / d x_d
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        sx += gv[d] * (H[2][d][1] - H[1][d][2]);
        sy += gv[d] * (H[0][d][2] - H[2][d][0]);
        sz += gv[d] * (H[1][d][0] - H[0][d][1]);
      }
    }
    far_u[3 * j] = ux * c4;
    far_u[3 * j + 1] = uy * c4;
    far_u[3 * j + 2] = uz * c4;
    far_s[3 * j] = sx * c4;
    far_s[3 * j + 1] = sy * c4;
    far_s[3 * j + 2] = sz * c4;
  }
}

}  // namespace

int downward_pass(fmm_plan p, int64_t n, cudaStream_t s) {
  const int P = p->P;
  for (int l = 1; l < p->nlevels; ++l) {
    int lb = p->level_begin[l], le = p->level_begin[l + 1];
    ++g_launches;
    k_l2l<<<le - lb, 128, 3 * P * sizeof(float), s>>>(lb, p->c_parent.as<int>(), p->c_key.as<uint64_t>(),
                                                      p->l2l_T.as<float>(), P, p->L.as<float>());
  }
  FMM_CUDA_TRY(cudaGetLastError());
  FMM_TRY(p->far_u.ensure((size_t)n * 3 * sizeof(float)));
  FMM_TRY(p->far_s.ensure((size_t)n * 3 * sizeof(float)));
  ++g_launches;
  k_l2p<<<(unsigned)p->nleaves, 64, (2 * 15 + 3) * P * sizeof(float), s>>>(
      p->leaves.as<int>(), p->c_begin.as<int>(), p->c_end.as<int>(), p->c_level.as<int>(), p->c_center.as<double>(),
      p->batched ? p->seg_box.as<double>() : p->scal.as<double>(), p->batched ? p->c_seg.as<int>() : nullptr,
      p->sortA.as<float4>(), p->sortB.as<float4>(), p->L.as<float>(), p->l2p_tab.as<int4>(),
      p->prm.p, (p->prm.outputs & FMM_OUT_STRETCHING_TRANSPOSE) ? 1 : 0, p->far_u.as<float>(), p->far_s.as<float>());
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

}  // namespace fmm
