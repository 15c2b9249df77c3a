// Periodic lattice operator (Sec. 3.5) built on the device in FP64.
//
// The 27 explicit images go through the traversal; beyond them the lattice of
// periodic copies acts on the root multipole through one P x P operator A:
//   A = sum_{lev=1}^{images-1} Ring(3^(lev-1)) . S_lev,
// where Ring(s) is the sum of the M2L operators from the 702 super-cells of
// side s (in root units) at offsets {-4..4}^3 \ {-1..1}^3 (times s) to the
// root, and S_lev the M2M that builds the level-(lev-1) super-cell multipole
// from the root's: S_1 = I, S_{lev+1} = S3 . S_lev, S3 the sum of the M2M
// operators of the 27 copies (offsets {-1,0,1}^3 in child units, scale 1/3).
// Every sum runs in a fixed order (offsets in (ox, oy, oz) order, products
// as plain loops), so the operator is the same bit for bit on every build.
#include <algorithm>

#include "fmm_internal.cuh"
#include "harmonics.cuh"

namespace fmm {

namespace {

constexpr int kGroup = 64;  // ring offsets evaluated per pass

// The 702 ring offsets in (ox, oy, oz) order.
__device__ __forceinline__ void ring_offset(int q, int& ox, int& oy, int& oz) {
  int c = -1;
  for (int x = -4; x <= 4; ++x)
    for (int y = -4; y <= 4; ++y)
      for (int z = -4; z <= 4; ++z) {
        if (max(abs(x), max(abs(y), abs(z))) <= 1) continue;
        if (++c == q) {
          ox = x;
          oy = y;
          oz = z;
          return;
        }
      }
}

// (n, m, part) of real-packed index r: degree n owns [n^2, (n+1)^2) as
// [Re m0, Re m1, Im m1, ...].
__device__ __forceinline__ void unpack_idx(int r, int& n, int& m, int& part) {
  n = (int)sqrtf((float)r);
  while (n * n > r) --n;
  while ((n + 1) * (n + 1) <= r) ++n;
  const int o = r - n * n;
  m = (o + 1) / 2;
  part = (o == 0) ? 0 : ((o - 1) & 1);
}

// parts[g][e] = entry e of the M2L operator of ring offset q0 + g (side s):
// translation tau = -o s (root units), source/target scale ratio s.
__global__ void k_ring_parts(int p, int q0, int nq, double s, double* __restrict__ parts) {
  __shared__ cd I[(2 * kPMax - 1) * (2 * kPMax) / 2];
  const int g = blockIdx.x;
  if (g >= nq) return;
  int ox, oy, oz;
  ring_offset(q0 + g, ox, oy, oz);
  if (threadIdx.x == 0) irregular_table_d(-ox * s, -oy * s, -oz * s, 2 * p - 1, I);
  __syncthreads();
  const int P = p * p;
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    int n, m, po, j, k, pi;
    unpack_idx(e / P, n, m, po);
    unpack_idx(e % P, j, k, pi);
    double rj = 1.0;
    for (int t = 0; t < j; ++t) rj *= s;
    parts[(size_t)g * P * P + e] = m2l_entry(I, n, m, po, j, k, pi, rj);
  }
}

// ring[e] += parts[0][e] + parts[1][e] + ... (in offset order)
__global__ void k_ring_accumulate(const double* __restrict__ parts, int nq, int PP, double* __restrict__ ring) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= PP) return;
  double acc = ring[e];
  for (int g = 0; g < nq; ++g) acc += parts[(size_t)g * PP + e];
  ring[e] = acc;
}

// S3 = sum over the 27 copies of the M2M from a cell to the super-cell of
// three times its side (child offset o in child units, scale ratio 1/3).  One
// thread per output (n, m >= 0): it owns both real rows of that coefficient.
__global__ void k_super_m2m(int p, double* __restrict__ S3) {
  const int P = p * p;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p * (p + 1) / 2) return;
  int n = 0;
  while ((n + 1) * (n + 2) / 2 <= idx) ++n;
  const int m = idx - n * (n + 1) / 2;
  cd R[kPMax * (kPMax + 1) / 2];
  double ratio_n = 1.0;
  for (int t = 0; t < n; ++t) ratio_n /= 3.0;
  const int row_re = ridx(n, m, 0), row_im = m > 0 ? ridx(n, m, 1) : -1;
  for (int c = 0; c < P; ++c) {
    S3[(size_t)row_re * P + c] = 0.0;
    if (row_im >= 0) S3[(size_t)row_im * P + c] = 0.0;
  }
  for (int ox = -1; ox <= 1; ++ox)
    for (int oy = -1; oy <= 1; ++oy)
      for (int oz = -1; oz <= 1; ++oz) {
        regular_table_d((double)ox, (double)oy, (double)oz, p, R);
        for (int k = 0; k <= n; ++k)
          for (int l = -k; l <= k; ++l) {
            if (abs(m - l) > n - k) continue;
            const double w = ratio_n * nu_d(n, m) / (nu_d(k, l) * nu_d(n - k, m - l));
            const cd c = cscale(cconj(harm_get(R, k, l)), w);
            // output (n, m) += c * X_{n-k}^{m-l}, X^{-k'} = (-1)^k' conj(X^k')
            const int j = n - k, kk = m - l, ak = kk < 0 ? -kk : kk;
            const double sgn = (kk < 0 && (ak & 1)) ? -1.0 : 1.0;
            const bool conj_in = kk < 0;
            const double br = conj_in ? -1.0 : 1.0;
            const cd ca = {c.re * sgn, c.im * sgn};
            const cd cb = {-c.im * sgn * br, c.re * sgn * br};
            const int col_a = ridx(j, ak, 0);
            S3[(size_t)row_re * P + col_a] += ca.re;
            if (row_im >= 0) S3[(size_t)row_im * P + col_a] += ca.im;
            if (ak > 0) {
              const int col_b = ridx(j, ak, 1);
              S3[(size_t)row_re * P + col_b] += cb.re;
              if (row_im >= 0) S3[(size_t)row_im * P + col_b] += cb.im;
            }
          }
      }
}

// C = A . B for P x P row-major FP64 matrices (plain loop over k in order).
__global__ void k_dgemm(const double* __restrict__ A, const double* __restrict__ B, int P, double* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P * P) return;
  const int i = e / P, j = e % P;
  double acc = 0.0;
  for (int k = 0; k < P; ++k) acc += A[(size_t)i * P + k] * B[(size_t)k * P + j];
  C[e] = acc;
}

__global__ void k_identity(int P, double* __restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < P * P) S[e] = (e / P == e % P) ? 1.0 : 0.0;
}

__global__ void k_add(const double* __restrict__ x, int n, double* __restrict__ y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] += x[e];
}

}  // namespace

// Builds the lattice operator into A (device, P x P FP64) on stream s, with
// scratch from the caller: 5 P x P matrices plus kGroup of them for the ring
// parts.  Synchronizes s (plan creation only).
int lattice_operator_device(int p, int images, double* A, cudaStream_t s) {
  const int P = p * p, PP = P * P;
  const int T = 256;
  const unsigned gpp = (unsigned)((PP + T - 1) / T);
  DBuf buf;  // released on every return path below
  const size_t mats = 5 + kGroup;
  FMM_TRY(buf.ensure(mats * (size_t)PP * sizeof(double)));
  double* S = buf.as<double>();
  double* S3 = S + PP;
  double* ring = S3 + PP;
  double* tmp = ring + PP;
  double* parts = tmp + 2 * (size_t)PP;
  int rc = FMM_OK;
  if (cudaMemsetAsync(A, 0, (size_t)PP * sizeof(double), s) != cudaSuccess) rc = FMM_E_CUDA;
  ++g_launches;
  k_identity<<<gpp, T, 0, s>>>(P, S);
  ++g_launches;
  k_super_m2m<<<(unsigned)((p * (p + 1) / 2 + 63) / 64), 64, 0, s>>>(p, S3);
  double side = 1.0;  // super-cell side / root side
  for (int lev = 1; lev < images && rc == FMM_OK; ++lev) {
    if (cudaMemsetAsync(ring, 0, (size_t)PP * sizeof(double), s) != cudaSuccess) rc = FMM_E_CUDA;
    for (int q0 = 0; q0 < 702 && rc == FMM_OK; q0 += kGroup) {
      const int nq = std::min(kGroup, 702 - q0);
      g_launches += 2;
      k_ring_parts<<<nq, T, 0, s>>>(p, q0, nq, side, parts);
      k_ring_accumulate<<<gpp, T, 0, s>>>(parts, nq, PP, ring);
    }
    g_launches += 4;
    k_dgemm<<<gpp, T, 0, s>>>(ring, S, P, tmp);  // contribution of this ring
    k_add<<<gpp, T, 0, s>>>(tmp, PP, A);
    k_dgemm<<<gpp, T, 0, s>>>(S3, S, P, tmp);    // next super-cell
    if (cudaMemcpyAsync(S, tmp, (size_t)PP * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      rc = FMM_E_CUDA;
    side *= 3.0;
  }
  if (cudaGetLastError() != cudaSuccess && rc == FMM_OK) rc = FMM_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == FMM_OK) rc = FMM_E_CUDA;
  buf.release();
  return rc;
}

}  // namespace fmm
