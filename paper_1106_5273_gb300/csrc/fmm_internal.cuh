// Plan structure and the host-side entry points of each translation unit.
#pragma once

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "harmonics.cuh"
#include "primitives.cuh"

// Layout of the small device scalar block (doubles).
namespace fmm {
constexpr int kScalBox = 0;     // box_min[3], box_len
constexpr int kScalDipole = 4;  // dipole velocity correction [3] (double)
constexpr int kScalSigma = 8;   // float bits of max sigma (per-particle sigma)
constexpr int kScalCount = 16;  // u32 counters area
constexpr int kScalKeySpan = 40;  // AND and OR of the Morton keys (u64 each)
constexpr int kBatchBits = 16;  // Morton bits per axis of a batched evaluation (depth cap 16)
constexpr int kMaxBatch = 1 << (63 - 3 * kBatchBits);  // problems per batched evaluation

// Per-problem tables of a batched evaluation (one entry per non-empty problem).
struct SegMac {  // traversal: image shift and regularisation MAC (Sec. 3.3)
  double blen, smax;
  float blenf, ksf, slack0, pad;
};
struct SegP2P {  // near field: core width, class bounds, dipole correction
  float sigma, smax, blen, margin;
  float dip[3], pad;
};
// Host description of a batch (problems concatenated; nullptr = one problem).
struct SegSpec {
  int nseg;
  const int* h_off;      // [nseg+1] particle ranges of the problems
  const float* h_sigma;  // [nseg] uniform sigma per problem, or nullptr (per-particle sigma)
  const double* h_box;   // [nseg][4] periodic cubes (min xyz, side), or nullptr (free space)
};
}  // namespace fmm

// Plan: parameters, constant operator tables, and the grow-only workspace.
struct fmm_plan_s {
  fmm_params prm;
  int64_t n_max = 0;
  int P = 0;      // p^2 real coefficients per potential
  int Kpad = 0;   // unused (the BF16 layouts use 64 x m2l_kchunks(P))
  int device = 0;
  int timing = 0;
  int tc_ok = 0;  // tensor-core M2L usable for this p
  int tc_kind = 0;  // tensor-core element kind: 0 BF16x3, 1 TF32x3 (FMM_M2L_TENSOR_TF32)
  // batched evaluation (several independent problems in one tree forest)
  int batched = 0;         // 1 while the last evaluation was a batch
  int nseg = 1;            // problems (non-empty) of the last evaluation
  int kbits = fmm::kMaxLevel;  // Morton bits per axis
  fmm::DBuf seg_off;       // int32 [nseg+1]
  fmm::DBuf seg_box;       // double [nseg][4]
  fmm::DBuf seg_sig;       // float [nseg] uniform sigma (batch with uniform sigma)
  fmm::DBuf seg_smax;      // u32 float bits [nseg] largest sigma
  fmm::DBuf seg_mac;       // SegMac [nseg]
  fmm::DBuf seg_p2p;       // SegP2P [nseg]
  fmm::DBuf c_seg;         // int32 problem of each cell
  void* seg_pinned = nullptr;  // host staging of the problem tables
  size_t seg_pinned_bytes = 0;
  // constant operator tables (device)
  fmm::DBuf m2m_T;    // [8][P(k)][P(r)] FP32 transposed M2M matrices by child octant
  fmm::DBuf l2l_T;    // [8][P(k)][P(r)] FP32 transposed L2L matrices by child octant
  fmm::DBuf l2p_tab;  // [5][P] int4 L2P gather table (indices into L~, signed weights)
  fmm::DBuf lattice;  // [P][P] FP64 periodic lattice operator (row = output)
  // particles
  fmm::DBuf keys0, keys1, vals0, vals1;  // radix sort ping-pong
  uint64_t* skeys = nullptr;             // sorted keys (points into keys0/keys1)
  uint32_t* sidx = nullptr;              // sorted position -> input index
  fmm::DBuf sortA, sortB;                // float4 (x,y,z,sigma), (gx,gy,gz,0) in sorted order
  fmm::DBuf far_u, far_s;                // [n][3] far field, sorted order
  fmm::DBuf leaf_of;                     // [n]
  fmm::DBuf in_pos, in_gam, in_sig, out_vel, out_dg;  // staging of the _host entry point
  fmm::DBuf t_pos, t_gam, t_sig, t_vel;                // sources + zero-strength targets (fmm_eval_targets)
  // cells
  fmm::DBuf c_begin, c_end, c_level, c_parent, c_child, c_nchild;  // int32
  fmm::DBuf c_key;                                                  // u64 level-local Morton index
  fmm::DBuf c_center, c_radius2, c_radius;                          // double[3], u64 bits, double
  fmm::DBuf c_cf;                                                   // float4 (centre, radius) rounded to FP32
  fmm::DBuf c_tile;                                                 // int32 tile*64+slot of each cell
  fmm::DBuf tile_cells;                                             // cell of each (tile, slot) position
  fmm::DBuf c_ijk;       // uint64 integer cell coordinates, 21 bits per axis
  fmm::DBuf tile_first;  // int32 [ntiles+1]: tile t = tile_cells[tile_first[t] .. tile_first[t+1])
  fmm::DBuf tile_groups; // int32 (level, octant) cell counts, then cell and tile offsets of the groups
  fmm::DBuf leaves;                                                 // leaf cell ids
  fmm::DBuf M, L;                                                   // [cells][3][P] FP32
  fmm::DBuf Mbf;  // [cells][hi/lo][3][K chunks x 128 bytes] BF16 or TF32 hi/lo
  // traversal
  fmm::DBuf fr0, fr1;                                 // frontier int4 (a,b,o,0)
  fmm::DBuf tcount, tmask, tscan0, tscan1, tscan2;    // per-item scratch
  fmm::DBuf p2p_raw, m2l_raw;                         // int4 (a,b,o,0)
  fmm::DBuf lk0, lk1, lv0, lv1;                       // list sort ping-pong
  fmm::DBuf p2p_sorted, p2p_off;                      // int2 (b,o) by leaf, CSR offsets per leaf
  fmm::DBuf m2l_key, m2l_slot, ukeys;                 // per pair key, slot; unique keys
  fmm::DBuf T32, Tbf;                                 // M2L operator cache [slot]: FP32, BF16 hi/lo
  std::unordered_map<uint64_t, int> tcache;           // translation key -> cache slot
  int64_t tcache_cap = 0;
  fmm::DBuf tmiss_keys, tmiss_slots, tslot_map;       // keys to build, their slots; unique key -> slot
  std::vector<uint64_t> h_keys;
  std::vector<int> h_map;
  int64_t n_built = 0;                                // operators built by the last evaluation
  fmm::DBuf st_tile, st_slot, st_src, tile_range;     // M2L steps
  fmm::DBuf bin_flag, bin_scan, bin_flag2, bin_scan2;  // binned step build: key and bin tables
  fmm::DBuf st_ckey, st_fkey;                         // compact / full translation key per step
  fmm::DBuf m2l_items, m2l_partial;                   // M2L work items (+ split list); partial sums
  // scratch
  fmm::DBuf scan_tmp, sort_hist;
  fmm::DBuf scal;   // small scalars (see kScal*)
  fmm::DBuf flags;  // int error flags
  void* pinned = nullptr;  // host pinned scratch (counts)
  // host mirror of the last tree / lists
  std::vector<int> level_begin;  // cells of level l: [level_begin[l], level_begin[l+1])
  int64_t ncells = 0, nleaves = 0, ntiles = 0;
  int nlevels = 0;
  double cf_margin = 0.0;  // rounding margin of the FP32 cell copies (2e-6 x largest coordinate)
  int64_t n_p2p = 0, n_m2l = 0, n_keys = 0, n_steps = 0, p2p_pairs = 0;
  int64_t last_n = 0;
  int last_tc = 0;
  int m2l_stage_chunks = 0;  // K chunks per stage of the last tensor-core M2L
  fmm::DBuf dip_part;        // partial sums of the dipole term (written beside the traversal)
  // tree reuse (fmm_eval_strengths): set by a successful full evaluation of
  // the plan's own particles; epoch counts full evaluations (a captured graph
  // is valid only within the epoch it was captured in)
  int reuse_ok = 0;
  int reuse_ps = 0;         // the last evaluation had a per-particle sigma array
  float reuse_sig_u = 0.f;  // its uniform sigma
  double reuse_smax = 0.0;  // its largest sigma
  int64_t epoch = 0;
  // list capacities the next traversal starts from (0: from the cell count);
  // a traversal whose lists outgrow them grows them and runs again
  int64_t cap_fr0 = 0, cap_m0 = 0, cap_p0 = 0;
  int64_t trav_runs = 0;  // traversal launches of the last evaluation
  int64_t hw_fr = 0, hw_m = 0, hw_p = 0;  // list sizes the plan's evaluations needed (+1/8)
  fmm_stats stats;
  cudaEvent_t ev[8];
  int have_events = 0;
  // the upward pass runs on this plan stream while the traversal runs on the
  // caller's stream (both read only the tree); fork / join by events
  cudaStream_t s_up = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace fmm {
// tree.cu
int grow_cells(fmm_plan p, int64_t need, cudaStream_t s);
int build_tree(fmm_plan p, int64_t n, const float* pos, const float* gam, const float* sig, float sig_u,
               cudaStream_t s);
int upload_segments(fmm_plan p, const SegSpec& sg, cudaStream_t s);
int build_forest(fmm_plan p, int64_t n, const float* pos, const float* gam, const float* sig, const SegSpec& sg,
                 cudaStream_t s);
// operators.cu
int build_constant_operators(fmm_plan p);
int build_m2l_operators(fmm_plan p, cudaStream_t s);
int apply_lattice(fmm_plan p, cudaStream_t s);
int lattice_operator_host(int p, int images, double* out);
// lattice.cu
int lattice_operator_device(int p, int images, double* A, cudaStream_t s);
// upward.cu
int upward_pass(fmm_plan p, cudaStream_t s);
int dipole_pass(fmm_plan p, int64_t n, cudaStream_t s);
// traverse.cu
int traverse(fmm_plan p, double sigma_max_host, cudaStream_t s);
// per-problem MAC and near-field tables of a batch (after the forest is built)
int segment_tables(fmm_plan p, int per_particle_sigma, cudaStream_t s);
// m2l.cu
int m2l_simt(fmm_plan p, cudaStream_t s);
int m2l_tensor(fmm_plan p, cudaStream_t s);
// downward.cu
int downward_pass(fmm_plan p, int64_t n, cudaStream_t s);
// reuse.cu
int eval_strengths(fmm_plan p, const float* gam, float* vel, float* dg, cudaStream_t s);
// p2p.cu
int p2p_near(fmm_plan p, int64_t n, float sig_u, int per_particle_sigma, double smax, float* vel, float* dg,
             cudaStream_t s);
int p2p_direct_all(int64_t n, const float* pos, const float* gam, const float* sig, float sig_u, float* vel,
                   float* dg, cudaStream_t s);
}  // namespace fmm

namespace fmm {
// M2L translation key (level-independent thanks to the cell-size scaling):
// delta = level(target) - level(source); t = 2 (c_t - c_s - o L) / a_f with
// a_f the side of the finer of the two cells (an integer vector).
// Bits: [57,63) delta+32, [38,57) tx, [19,38) ty, [0,19) tz (two's complement).
constexpr int kKeyBits = 19;
constexpr long long kKeyLim = (1ll << (kKeyBits - 1)) - 1;

__host__ __device__ inline uint64_t m2l_key_encode(int delta, long long tx, long long ty, long long tz) {
  const uint64_t mask = (1ull << kKeyBits) - 1ull;
  return ((uint64_t)(delta + 32) << 57) | (((uint64_t)tx & mask) << 38) | (((uint64_t)ty & mask) << 19) |
         ((uint64_t)tz & mask);
}

__host__ __device__ inline long long key_field(uint64_t key, int shift) {
  long long v = (long long)((key >> shift) & ((1ull << kKeyBits) - 1ull));
  if (v >= (1ll << (kKeyBits - 1))) v -= (1ll << kKeyBits);
  return v;
}

// delta and tau = (c_t - c_s)/a_t (target-cell units); a_s/a_t = 2^delta.
__host__ __device__ inline void m2l_key_decode(uint64_t key, int* delta, double tau[3]) {
  int d = (int)(key >> 57) - 32;
  *delta = d;
  double f = 0.5 * (d < 0 ? ldexp(1.0, d) : 1.0);
  tau[0] = (double)key_field(key, 38) * f;
  tau[1] = (double)key_field(key, 19) * f;
  tau[2] = (double)key_field(key, 0) * f;
}

// K chunks of 64 coefficients (4 MMA K-steps of 16) covering P inputs.
// Tensor-core M2L element kinds: 0 = BF16 (kind::f16, K step 16), 1 = TF32
// (kind::tf32, K step 8).  A K chunk is one 128-byte row of either: 64 BF16 or
// 32 TF32 values, 4 K steps.
__host__ __device__ inline int m2l_kstep(int kind) { return kind ? 8 : 16; }
__host__ __device__ inline int m2l_kchunks(int P, int kind = 0) {
  return ((P + m2l_kstep(kind) - 1) / m2l_kstep(kind) + 3) / 4;
}
// K chunks of the BF16 tensor-core M2L that take all three split products.
// Under the MAC (R_A + R_B < theta |X_A - X_B|) the M2L terms of source
// degree j sum to at most theta^j / (1 - theta) of the leading 1/|X_A - X_B|
// term.  BF16 chunks from the second on hold degrees >= 8 (64 coefficients
// per chunk), so one hi x hi product there (relative error <= 2^-8) adds at
// most 2^-8 theta^8 / (1 - theta) of the leading term: <= 7e-6 for
// theta <= 0.42, whose theta^8 <= 2^-10.  Otherwise, and for TF32, every
// chunk takes three products.
__host__ __device__ inline int m2l_split_chunks(int P, int kind, float theta, bool full) {
  const int nkc = m2l_kchunks(P, kind);
  const float t2 = theta * theta, t8 = t2 * t2 * t2 * t2;
  return (kind == 0 && !full && t8 <= 1.0f / 1024.0f) ? 1 : nkc;
}
// Blocks of 128 output rows (one MMA M) covering P outputs.
__host__ __device__ inline int m2l_rowblocks(int P) { return (P + 127) / 128; }

// Level / tile layout of the current tree, passed to kernels by value.
}  // namespace fmm
