// Translation operators as real matrices on the real-packed coefficients.
//
// Sec. 3.1: M2M, M2L, L2L of the spherical-harmonic Laplace expansions
// (formulas in harmonics.cuh).  Octree children sit at beta = (+-1/2)^3 in
// child units with scale ratio 1/2, so M2M and L2L reduce to 8 fixed matrices
// per p, built here once in FP64 on the host.  Each distinct M2L translation
// (level difference, offset; see m2l_key_* in traverse.cu) becomes one P x P
// matrix built in FP64 on the device per evaluation.  The periodic far field
// (Sec. 3.5) is one FP64 P x P operator on the root multipole: images-1
// rings of 702 super-cells, each ring the M2L sum from offsets
// {-4..4}^3 \ {-1..1}^3, the next super-cell the M2M sum of 27 copies.
#include <complex>
#include <cstring>

#include "fmm_internal.cuh"
#include <cuda_bf16.h>

namespace fmm {

namespace {

using Mat = std::vector<double>;

// Y_n^m (m >= 0) += c * X_j^k  (conj_in: c * conj(X_j^k)), X_j^{-k} = (-1)^k conj(X_j^k).
void add_term(Mat& A, int P, int n, int m, int j, int k, cd c, bool conj_in) {
  int ak = k < 0 ? -k : k;
  double sgn = (k < 0 && (ak & 1)) ? -1.0 : 1.0;
  bool conj_total = (k < 0) != conj_in;
  double br = conj_total ? -1.0 : 1.0;
  cd ca = {c.re * sgn, c.im * sgn};
  cd cb = {-c.im * sgn * br, c.re * sgn * br};
  int row_re = ridx(n, m, 0);
  int col_a = ridx(j, ak, 0);
  A[(size_t)row_re * P + col_a] += ca.re;
  if (m > 0) A[(size_t)ridx(n, m, 1) * P + col_a] += ca.im;
  if (ak > 0) {
    int col_b = ridx(j, ak, 1);
    A[(size_t)row_re * P + col_b] += cb.re;
    if (m > 0) A[(size_t)ridx(n, m, 1) * P + col_b] += cb.im;
  }
}

Mat m2m_matrix(int p, const double beta[3], double ratio) {
  const int P = p * p;
  Mat A((size_t)P * P, 0.0);
  std::vector<cd> R(kPMax * (kPMax + 1) / 2);
  regular_table_d(beta[0], beta[1], beta[2], p, R.data());
  for (int n = 0; n < p; ++n)
    for (int m = 0; m <= n; ++m)
      for (int k = 0; k <= n; ++k)
        for (int l = -k; l <= k; ++l) {
          if (std::abs(m - l) > n - k) continue;
          double w = pow(ratio, n) * nu_d(n, m) / (nu_d(k, l) * nu_d(n - k, m - l));
          cd c = cscale(cconj(harm_get(R.data(), k, l)), w);
          add_term(A, P, n, m, n - k, m - l, c, false);
        }
  return A;
}

Mat l2l_matrix(int p, const double beta[3], double ratio) {
  const int P = p * p;
  Mat A((size_t)P * P, 0.0);
  std::vector<cd> R(kPMax * (kPMax + 1) / 2);
  regular_table_d(beta[0], beta[1], beta[2], p, R.data());
  for (int n = 0; n < p; ++n)
    for (int m = 0; m <= n; ++m)
      for (int k = 0; k < p - n; ++k)
        for (int l = -k; l <= k; ++l) {
          if (std::abs(m + l) > n + k) continue;
          double w = pow(ratio, n + k + 1) * nu_d(n + k, m + l) / (nu_d(n, m) * nu_d(k, l));
          cd c = cscale(harm_get(R.data(), k, l), w);
          add_term(A, P, n, m, n + k, m + l, c, false);
        }
  return A;
}

Mat m2l_matrix(int p, const double tau[3], double ratio) {
  const int P = p * p;
  Mat A((size_t)P * P, 0.0);
  const int D = 2 * p - 1;
  std::vector<cd> I(D * (D + 1) / 2);
  irregular_table_d(tau[0], tau[1], tau[2], D, I.data());
  for (int n = 0; n < p; ++n)
    for (int m = 0; m <= n; ++m)
      for (int j = 0; j < p; ++j)
        for (int k = -j; k <= j; ++k) {
          double w = ((n & 1) ? -1.0 : 1.0) * pow(ratio, j) / (nu_d(n, m) * nu_d(j, k));
          cd c = cscale(cconj(harm_get(I.data(), j + n, k + m)), w);
          add_term(A, P, n, m, j, k, c, true);
        }
  return A;
}

Mat matmul(const Mat& A, const Mat& B, int P) {
  Mat C((size_t)P * P, 0.0);
  for (int i = 0; i < P; ++i)
    for (int k = 0; k < P; ++k) {
      double a = A[(size_t)i * P + k];
      if (a == 0.0) continue;
      for (int j = 0; j < P; ++j) C[(size_t)i * P + j] += a * B[(size_t)k * P + j];
    }
  return C;
}

// Lattice operator: L~_root += A_lat M~_root (root side = box length).
Mat lattice_matrix(int p, int images) {
  const int P = p * p;
  Mat A((size_t)P * P, 0.0);
  Mat S((size_t)P * P, 0.0);  // M2M of level-(lev-1) super-cell from the root
  for (int i = 0; i < P; ++i) S[(size_t)i * P + i] = 1.0;
  // one-level super-cell M2M: 27 copies at offsets o (child units), ratio 1/3
  Mat S3((size_t)P * P, 0.0);
  for (int ox = -1; ox <= 1; ++ox)
    for (int oy = -1; oy <= 1; ++oy)
      for (int oz = -1; oz <= 1; ++oz) {
        double b[3] = {(double)ox, (double)oy, (double)oz};
        Mat T = m2m_matrix(p, b, 1.0 / 3.0);
        for (size_t q = 0; q < T.size(); ++q) S3[q] += T[q];
      }
  double scale = 1.0;  // super-cell side / root side
  for (int lev = 1; lev < images; ++lev) {
    Mat ring((size_t)P * P, 0.0);
    for (int ox = -4; ox <= 4; ++ox)
      for (int oy = -4; oy <= 4; ++oy)
        for (int oz = -4; oz <= 4; ++oz) {
          if (std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz))) <= 1) continue;
          double tau[3] = {-ox * scale, -oy * scale, -oz * scale};
          Mat T = m2l_matrix(p, tau, scale);
          for (size_t q = 0; q < T.size(); ++q) ring[q] += T[q];
        }
    Mat contrib = matmul(ring, S, P);
    for (size_t q = 0; q < A.size(); ++q) A[q] += contrib[q];
    S = matmul(S3, S, P);
    scale *= 3.0;
  }
  return A;
}

// ---- device: M2L operator per translation key

// Round an FP32 value to TF32 (10 stored mantissa bits, to nearest, ties to
// even) in its 32-bit container; the low 13 bits end up zero.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;  // inf / nan
  u += 0x0FFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xFFFFE000u);
}

// kind 0: BF16 tiles [key][hi/lo][nkc K chunks of 64][rows][64];
// kind 1: TF32 tiles [key][hi/lo][nkc K chunks of 32][rows][32]; both 128-byte
// rows with 16-byte groups in the 128-byte swizzle order (group j at j ^ (row & 7)).
__global__ void k_build_m2l(const uint64_t* __restrict__ keys, const int* __restrict__ slots, int nkeys, int p,
                            float* __restrict__ T32, uint8_t* __restrict__ Tb, int nkc, int kind) {
  __shared__ cd I[(2 * kPMax - 1) * (2 * kPMax) / 2];
  __shared__ double nu[kNCoefMax];
  __shared__ double rp[kPMax];
  __shared__ int nmp[kNCoefMax];  // real index -> (n, m, part) packed
  const int kid = blockIdx.x;
  if (kid >= nkeys) return;
  const int key_id = slots[kid];  // cache slot written by this block
  const int P = p * p;
  uint64_t key = keys[kid];
  int delta;
  double tau[3];
  m2l_key_decode(key, &delta, tau);
  if (threadIdx.x == 0) irregular_table_d(tau[0], tau[1], tau[2], 2 * p - 1, I);
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    int n = (int)sqrtf((float)r);
    while (n * n > r) --n;
    while ((n + 1) * (n + 1) <= r) ++n;
    int o = r - n * n;
    int m = (o + 1) / 2, part = (o == 0) ? 0 : ((o - 1) & 1);
    nmp[r] = (n << 16) | (m << 8) | part;
    nu[r] = nu_d(n, m);
  }
  if (threadIdx.x < (unsigned)p) rp[threadIdx.x] = ldexp(1.0, delta * (int)threadIdx.x);
  const int rows = 128 * m2l_rowblocks(P);  // output rows of the BF16 tiles
  const size_t chunk_bytes = (size_t)rows * 128;
  if (nkc) {  // zero this slot's tiles (padding rows and columns stay zero)
    uint4* z = reinterpret_cast<uint4*>(Tb + (size_t)key_id * 2 * nkc * chunk_bytes);
    for (size_t i = threadIdx.x; i < 2 * nkc * chunk_bytes / 16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    int r = e / P, c = e % P;
    int a = nmp[r], b = nmp[c];
    int n = a >> 16, m = (a >> 8) & 0xff, po = a & 1;
    int j = b >> 16, k = (b >> 8) & 0xff, pi = b & 1;
    double s = ((n & 1) ? -1.0 : 1.0) * rp[j] / (nu[r] * nu[c]);
    cd A = cconj(harm_get(I, j + n, k + m));
    cd B = {0.0, 0.0};
    if (k > 0) {
      B = cconj(harm_get(I, j + n, m - k));
      if (k & 1) B = {-B.re, -B.im};
    }
    double v;
    if (pi == 0) v = po == 0 ? s * (A.re + B.re) : s * (A.im + B.im);
    else v = po == 0 ? -s * (B.im - A.im) : s * (B.re - A.re);
    if (!nkc) T32[(size_t)key_id * P * P + e] = (float)v;  // FP32 copy for the SIMT path only
    if (nkc && kind == 0) {
      __nv_bfloat16* Tbf = reinterpret_cast<__nv_bfloat16*>(Tb);
      __nv_bfloat16 hi = __double2bfloat16(v);
      __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
      const int kc = c >> 6, j = (c & 63) >> 3, el = c & 7;
      const size_t within = (size_t)r * 64 + (size_t)(((j ^ (r & 7)) << 3) + el);
      Tbf[(((size_t)key_id * 2 + 0) * nkc + kc) * ((size_t)rows * 64) + within] = hi;
      Tbf[(((size_t)key_id * 2 + 1) * nkc + kc) * ((size_t)rows * 64) + within] = lo;
    } else if (nkc) {
      float* Ttf = reinterpret_cast<float*>(Tb);
      const float hi = round_tf32((float)v);
      const float lo = round_tf32((float)(v - (double)hi));
      const int kc = c >> 5, j = (c & 31) >> 2, el = c & 3;
      const size_t within = (size_t)r * 32 + (size_t)(((j ^ (r & 7)) << 2) + el);
      Ttf[(((size_t)key_id * 2 + 0) * nkc + kc) * ((size_t)rows * 32) + within] = hi;
      Ttf[(((size_t)key_id * 2 + 1) * nkc + kc) * ((size_t)rows * 32) + within] = lo;
    }
  }
}

// One CTA per root cell (one per problem; the normalised operator does not
// depend on the cube size): L[root][c][r] += sum_k A[r][k] M[root][c][k]
__global__ void k_apply_lattice(const double* __restrict__ A, int P, float* __restrict__ L, const float* __restrict__ M) {
  const size_t root = (size_t)blockIdx.x * 3 * P;
  for (int e = threadIdx.x; e < 3 * P; e += blockDim.x) {
    int c = e / P, r = e % P;
    double acc = 0.0;
    for (int k = 0; k < P; ++k) acc += A[(size_t)r * P + k] * (double)M[root + c * P + k];
    L[root + c * P + r] += (float)acc;
  }
}

}  // namespace

int build_constant_operators(fmm_plan p) {
  const int pp = p->prm.p, P = pp * pp;
  std::vector<float> m2mT((size_t)8 * P * P), l2lT((size_t)8 * P * P);
  for (int oct = 0; oct < 8; ++oct) {
    double beta[3] = {(oct & 4) ? 0.5 : -0.5, (oct & 2) ? 0.5 : -0.5, (oct & 1) ? 0.5 : -0.5};
    Mat A = m2m_matrix(pp, beta, 0.5);
    Mat B = l2l_matrix(pp, beta, 0.5);
    for (int r = 0; r < P; ++r)
      for (int k = 0; k < P; ++k) {
        m2mT[(size_t)oct * P * P + (size_t)k * P + r] = (float)A[(size_t)r * P + k];
        l2lT[(size_t)oct * P * P + (size_t)k * P + r] = (float)B[(size_t)r * P + k];
      }
  }
  FMM_TRY(p->m2m_T.ensure(m2mT.size() * sizeof(float)));
  FMM_TRY(p->l2l_T.ensure(l2lT.size() * sizeof(float)));
  FMM_CUDA_TRY(cudaMemcpy(p->m2m_T.ptr, m2mT.data(), m2mT.size() * sizeof(float), cudaMemcpyHostToDevice));
  FMM_CUDA_TRY(cudaMemcpy(p->l2l_T.ptr, l2lT.data(), l2lT.size() * sizeof(float), cudaMemcpyHostToDevice));
  // L2P weights for the 5 outputs (n',m') in {(1,0),(1,1),(2,0),(2,1),(2,2)}
  // over inputs (k,l), |l| <= k, index k^2 + k + l:  nu_{n'+k}^{m'+l} / nu_k^l
  const int outs[5][2] = {{1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
  std::vector<float> w((size_t)5 * P, 0.f);
  for (int o = 0; o < 5; ++o)
    for (int k = 0; k < pp; ++k)
      for (int l = -k; l <= k; ++l) {
        int n2 = outs[o][0], m2 = outs[o][1];
        if (n2 + k > pp - 1 || std::abs(m2 + l) > n2 + k) continue;
        w[(size_t)o * P + k * k + k + l] = (float)(nu_d(n2 + k, m2 + l) / nu_d(k, l));
      }
  // The L2P gather table: entry o P + (k^2 + k + mm) of the leaf's derivative
  // coefficients D_o(k, mm) = c_re L~(i_re) + i c_im L~(i_im) (per potential),
  // with L~_N^M, N = n'_o + k, M = m'_o + mm read from the real-packed
  // storage (re at N^2 + (|M| ? 2|M| - 1 : 0), im at N^2 + 2|M|), the signs
  // of M < 0, the weight, and (-1)^m for mm = -m < 0 folded into
  // c_re, c_im (zero where N > p - 1 or the term has no imaginary part).
  std::vector<int4> tab((size_t)5 * P);
  for (int o = 0; o < 5; ++o)
    for (int k = 0; k < pp; ++k)
      for (int mm = -k; mm <= k; ++mm) {
        const int kk = k * k + k + mm, m = std::abs(mm);
        const int N = outs[o][0] + k, M = outs[o][1] + mm;
        int4 t = make_int4(0, 0, 0, 0);
        if (N <= pp - 1) {
          const float wv = w[(size_t)o * P + kk];
          const float sg = (mm < 0 && (m & 1)) ? -wv : wv;
          const int am = std::abs(M);
          float sre = 1.f, sim = am == 0 ? 0.f : 1.f;
          if (M < 0) {  // L~_N^{-|M|} = (-1)^|M| conj(L~_N^{|M|})
            sim = -sim;
            if (am & 1) {
              sre = -sre;
              sim = -sim;
            }
          }
          const float cre = sg * sre, cim = sg * sim;
          t.x = N * N + (am == 0 ? 0 : 2 * am - 1);
          t.y = am == 0 ? 0 : N * N + 2 * am;
          std::memcpy(&t.z, &cre, sizeof(float));
          std::memcpy(&t.w, &cim, sizeof(float));
        }
        tab[(size_t)o * P + kk] = t;
      }
  FMM_TRY(p->l2p_tab.ensure(tab.size() * sizeof(int4)));
  FMM_CUDA_TRY(cudaMemcpy(p->l2p_tab.ptr, tab.data(), tab.size() * sizeof(int4), cudaMemcpyHostToDevice));
  if (p->prm.periodic) {  // the lattice operator, in FP64 on the device
    FMM_TRY(p->lattice.ensure((size_t)P * P * sizeof(double)));
    FMM_TRY(lattice_operator_device(pp, p->prm.images, p->lattice.as<double>(), 0));
  }
  return FMM_OK;
}

// The lattice operator built on the host (the same sums in FP64 C++), kept to
// cross-check the device build (fmm_lattice_operator).
int lattice_operator_host(int p, int images, double* out) {
  Mat A = lattice_matrix(p, images);
  for (size_t q = 0; q < A.size(); ++q) out[q] = A[q];
  return FMM_OK;
}

__global__ void k_remap_slots(int* __restrict__ st_slot, int64_t ns, const int* __restrict__ map) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ns) st_slot[i] = map[st_slot[i]];
}

// M2L operators are constants of (translation key, p): the plan keeps them in a
// cache indexed by key and builds (in FP64, on the device) only the keys it has
// not seen; the step list is then re-pointed from unique-key index to slot.
int build_m2l_operators(fmm_plan p, cudaStream_t s) {
  const int P = p->P;
  p->n_built = 0;
  if (p->n_keys == 0) return FMM_OK;
  const int64_t nk = p->n_keys;
  p->h_keys.resize(nk);
  FMM_CUDA_TRY(cudaMemcpyAsync(p->h_keys.data(), p->ukeys.ptr, nk * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  // BF16 tiles only for the tensor-core path (the plan's M2L mode does not
  // change between evaluations)
  const int tc = p->last_tc;
  // bound the cache: start over when this evaluation's new operators would
  // take it past 1 << 16 (a cleared cache then holds exactly this evaluation's)
  {
    int64_t misses = 0;
    for (int64_t i = 0; i < nk; ++i) misses += p->tcache.count(p->h_keys[i]) ? 0 : 1;
    if ((int64_t)p->tcache.size() + misses > (1 << 16)) p->tcache.clear();
  }
  p->h_map.resize(nk);
  std::vector<uint64_t> miss_keys;
  std::vector<int> miss_slots;
  for (int64_t i = 0; i < nk; ++i) {
    auto it = p->tcache.find(p->h_keys[i]);
    if (it != p->tcache.end()) {
      p->h_map[i] = it->second;
    } else {
      int slot = (int)p->tcache.size();
      p->tcache.emplace(p->h_keys[i], slot);
      p->h_map[i] = slot;
      miss_keys.push_back(p->h_keys[i]);
      miss_slots.push_back(slot);
    }
  }
  const int64_t need = (int64_t)p->tcache.size();
  if (need > p->tcache_cap) {
    int64_t cap = std::max<int64_t>(need, p->tcache_cap * 2);
    if (!tc) FMM_TRY(p->T32.grow_copy((size_t)cap * P * P * sizeof(float), s));
    if (tc)
      FMM_TRY(p->Tbf.grow_copy((size_t)cap * 2 * m2l_kchunks(P, p->tc_kind) * 128 * m2l_rowblocks(P) * 128, s));
    p->tcache_cap = cap;
  }
  if (!miss_keys.empty()) {
    const int64_t nm = (int64_t)miss_keys.size();
    FMM_TRY(p->tmiss_keys.ensure(nm * sizeof(uint64_t)));
    FMM_TRY(p->tmiss_slots.ensure(nm * sizeof(int)));
    FMM_CUDA_TRY(cudaMemcpyAsync(p->tmiss_keys.ptr, miss_keys.data(), nm * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(p->tmiss_slots.ptr, miss_slots.data(), nm * sizeof(int), cudaMemcpyHostToDevice, s));
    ++g_launches;
    k_build_m2l<<<(unsigned)nm, 256, 0, s>>>(p->tmiss_keys.as<uint64_t>(), p->tmiss_slots.as<int>(), (int)nm,
                                             p->prm.p, p->T32.as<float>(), p->Tbf.as<uint8_t>(),
                                             tc ? m2l_kchunks(P, p->tc_kind) : 0, p->tc_kind);
    FMM_CUDA_TRY(cudaGetLastError());
    p->n_built = nm;
  }
  FMM_TRY(p->tslot_map.ensure(nk * sizeof(int)));
  FMM_CUDA_TRY(cudaMemcpyAsync(p->tslot_map.ptr, p->h_map.data(), nk * sizeof(int), cudaMemcpyHostToDevice, s));
  ++g_launches;
  k_remap_slots<<<(unsigned)((p->n_steps + 255) / 256), 256, 0, s>>>(p->st_slot.as<int>(), p->n_steps,
                                                                    p->tslot_map.as<int>());
  FMM_CUDA_TRY(cudaGetLastError());
  // the host vectors above are read by the copies before they change again
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  return FMM_OK;
}

int apply_lattice(fmm_plan p, cudaStream_t s) {
  if (!p->prm.periodic || p->prm.images <= 1) return FMM_OK;
  ++g_launches;
  k_apply_lattice<<<p->batched ? p->nseg : 1, 512, 0, s>>>(p->lattice.as<double>(), p->P, p->L.as<float>(),
                                                           p->M.as<float>());
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

}  // namespace fmm
