// Continuous-Galerkin apply with the interpolation products on the 5th-generation
// tensor cores (tcgen05, sm_103a), TF32 or BF16 operands with FP32 accumulation.
//
// The two dense contractions of Eq. 3 for a batch of 128 cells become GEMMs
// ("matrix-matrix product", Sec. 2.4, with the batch extended from 4 x n_lanes
// cells to 128 cells = the M of one tcgen05.mma):
//   GEMM 1:  G[128 x 3nq]  = U'[128 x nd-1] . E'^T   (E' = columns 1..nd-1 of E, Eq. 4;
//                                                     U'[m, j-1] = u_j - u_0 of cell m)
//   D_e:     Q[m, (q,k)]   = w_q k_q (M_e G[m, (q,0..2)])_k  per thread (row m)
//   GEMM 2:  Y'[128 x nd-1] = Q[128 x 3nq] . E',      y_0 = -sum_{j>=1} y_j
// Columns (q, k) of G and Q are stored in pairs of points, (x_q, x_q', y_q, y_q', z_q, z_q'),
// so that the metric step runs on packed FP32x2 instructions (grad_col).
// The difference form is E u_e rewritten with sum_j E_j = 0 (partition of
// unity); it is exact for exact tables and keeps rounded TF32/BF16 tables
// consistent (constants map to zero, operand error relative to the gradient).
//
// Data movement: each 128-cell tile carries the list of the distinct 16-byte
// groups (4 consecutive DoFs) that hold its unconstrained DoFs, in the order of
// their staging slots (sorted, then permuted inside windows of 8 to spread a
// warp's shared-memory accesses over the banks) and, per (cell, local node), a
// 16-bit position in the tile's staging.  Set-up numbers
// the DoFs by the set of tiles sharing them, so a tile's DoFs fill its groups
// densely (at P3 about 880 DoFs in 240 groups).  The values are gathered with
// one 16-byte cp.async per group, and the tile's contributions are pre-reduced
// in shared memory before one 16-byte vector atomic per group: about 11x fewer
// gather requests and L2 atomics than one per (cell, node) (the masked gather
// and the scatter of Sec. 2.4).
//
// A warpgroup of 128 threads owns one TMEM lane per cell and loops over tiles:
//   1. build row m of U' from the staged values, write it to shared memory;
//   2. one thread issues GEMM 1 (D in TMEM), commits to an mbarrier; meanwhile
//      the previous tile is scattered (step 5); then the warpgroup starts
//      copying the values of the tile after next and the list and node
//      indices of the one after that (cp.async, a ring of four stages);
//   3. each thread reads its row of G from TMEM in chunks of 16 points,
//      applies the metric in FP32 and writes Q back into TMEM (tcgen05.st);
//   4. one thread issues GEMM 2 with A = Q in TMEM; it runs while the next
//      tile's rows are built;
//   5. each thread reads its row of Y', pre-reduces it into shared memory,
//      and the warpgroup adds the tile's distinct values to y with atomics.
// Where TMEM admits at most three tiles per SM (P3, P4) and there is no coefficient, the
// warp-specialised kernel below takes step 5 off the compute warpgroups: a fourth warpgroup
// scatters every finished tile while they carry on with the next.
// Every wait on an MMA completion is bounded (about 1 s); on time-out the
// kernel records bit 0 in the status word and stops after freeing its TMEM.
//
// Shared-memory operand layout (K-major, no swizzle): a core matrix is 8 rows
// x 16 bytes, stored contiguously; row r, column k of an operand with R rows
// sits at  (k / KC) * LBO + (r / 8) * 128 + (r % 8) * 16 + (k % KC) * ES,
// KC = 16 / ES elements per core-matrix row, SBO = 128 (next 8 rows),
// LBO = (R / 8) * 128 (next 16-byte column block).  One MMA consumes K = 2 KC.
// The A operand of GEMM 2 lives in TMEM: lane m = row m, one 32-bit column
// per TF32 element or per pair of BF16 elements.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace tetmf {
namespace {

constexpr int kT = kTile;




// per-tile staging buffers: a ring of stages per warpgroup.  Four stages (tile t, values of t+1, values
// of t+2 in flight, tile t-1 being flushed and then the metadata of t+3) where TMEM keeps a CTA below
// four warpgroups, so that shared memory is left over; three (tile t, values of t+1 in flight, tile
// t-1 and then the metadata of t+2) where four warpgroups fit, which need the shared memory.
// lmax: the longest group list, a multiple of 4
template <int ND, int NQ, bool HAS_K>
struct Stage {
  uint32_t* lidx;   // [NDP / 2][128] pairs of 16-bit staging positions (node 2w low, 2w+1 high)
  int32_t* list;    // [lmax] distinct 16-byte groups of the tile
  float* vals;      // [4 lmax + 4] their values and the zero slot, then the tile's pre-reduced results
  float* kt;        // [128][NQ | 1] coefficient tile (HAS_K)
};

template <int ND, int NQ, bool HAS_K>
__host__ __device__ constexpr size_t stage_bytes(int lmax) {
  return size_t(round_up(ND, 2)) * kT * 2 + size_t(lmax) * 4 + (size_t(lmax) * 4 + 4) * 4 +
         (HAS_K ? size_t(kT) * (NQ | 1) * 4 : 0);
}

template <int ND, int NQ, bool HAS_K>
__device__ inline Stage<ND, NQ, HAS_K> stage_at(uint8_t* p, int lmax) {
  Stage<ND, NQ, HAS_K> st;
  st.lidx = reinterpret_cast<uint32_t*>(p);
  p += round_up(ND, 2) * kT * 2;
  st.list = reinterpret_cast<int32_t*>(p);
  p += size_t(lmax) * 4;
  st.vals = reinterpret_cast<float*>(p);
  p += (size_t(lmax) * 4 + 4) * 4;
  st.kt = HAS_K ? reinterpret_cast<float*>(p) : nullptr;
  return st;
}

// where a tile's group list starts and how long it is; loaded a tile ahead of its use, so that the
// copies below do not wait on the load
struct Span {
  int64_t o;
  int L;
};
__device__ inline Span load_span(const int64_t* __restrict__ tl_span, int64_t tile, int64_t ntiles) {
  if (tile >= ntiles) return Span{0, 0};
  return Span{__ldg(tl_span + 2 * tile), int(__ldg(tl_span + 2 * tile + 1))};
}
// the cell metric of row m of a tile (6 values), likewise loaded a tile ahead
struct Metric {
  float v[6];
};
__device__ inline Metric load_metric(const float* __restrict__ metric, int64_t tile, int64_t ntiles, int m) {
  Metric r;
  const float* mp = metric + (tile < ntiles ? tile : 0) * 6 * kT + m;
#pragma unroll
  for (int a = 0; a < 6; ++a) r.v[a] = __ldg(mp + a * kT);
  return r;
}

// the copies of a tile's list and node positions (and coefficients) into a stage; m = thread of the
// warpgroup
template <int ND, int NQ, bool HAS_K>
__device__ inline void meta_copies(const Stage<ND, NQ, HAS_K>& st, int m, int64_t tile, Span sp,
                                   const int32_t* __restrict__ tl_list, const uint16_t* __restrict__ tl_lidx,
                                   const float* __restrict__ kcoef, int64_t nc) {
  constexpr int NDP = round_up(ND, 2);
  const int32_t* src_list = tl_list + sp.o;  // 16-byte aligned, padded to a multiple of 4 entries
  for (int i = m; i < (sp.L + 3) / 4; i += kT) cp_async16(st.list + 4 * i, src_list + 4 * i);
  const uint8_t* li = reinterpret_cast<const uint8_t*>(tl_lidx + tile * NDP * kT);
  for (int i = m; i < NDP * kT * 2 / 16; i += kT) cp_async16(reinterpret_cast<uint8_t*>(st.lidx) + 16 * i, li + 16 * i);
  if constexpr (HAS_K) {
    const int64_t cell0 = tile * kT;
    const int64_t n = (nc - cell0 < kT ? nc - cell0 : kT) * NQ;
    const float* src = kcoef + cell0 * NQ;
    for (int i = m; i < int(n); i += kT) cp_async4(st.kt + (i / NQ) * (NQ | 1) + i % NQ, src + i);
  }
}

// copy a tile's list and node positions (and coefficients) into a stage, as one cp.async group
template <int ND, int NQ, bool HAS_K>
__device__ inline int issue_meta(const Stage<ND, NQ, HAS_K>& st, int m, int64_t tile, Span sp,
                                     const int32_t* __restrict__ tl_list,
                                     const uint16_t* __restrict__ tl_lidx, const float* __restrict__ kcoef,
                                     int64_t nc) {
  meta_copies<ND, NQ, HAS_K>(st, m, tile, sp, tl_list, tl_lidx, kcoef, nc);
  cp_async_commit();
  return sp.L;
}

// gather the values of a tile's groups (after its list has arrived) as one cp.async group: one
// 16-byte copy per group where u is 16-byte aligned and the group lies inside the vector (n DoFs),
// else the group's DoFs one by one (the vector's last, partial group)
template <int ND, int NQ, bool HAS_K>
__device__ inline void issue_gather(const Stage<ND, NQ, HAS_K>& st, int m, int L, const float* __restrict__ u,
                                    int64_t n, bool u16) {
  for (int i = m; i < L; i += kT) {
    const int64_t base = 4 * int64_t(st.list[i]);
    if (u16 && base + 4 <= n) {
      cp_async16(st.vals + 4 * i, u + base);
    } else {
      for (int e = 0; e < 4; ++e)
        if (base + e < n) cp_async4(st.vals + 4 * i + e, u + base + e);
    }
  }
  if (m == 0) *reinterpret_cast<float4*>(st.vals + 4 * L) = make_float4(0.f, 0.f, 0.f, 0.f);  // zero slot
  cp_async_commit();
}

// add a tile's pre-reduced groups to y: one 16-byte vector reduction (no return value) per group
// where y is 16-byte aligned and the group lies inside the vector, else one atomic per DoF
__device__ inline void flush_group(float* __restrict__ y, int32_t group, float4 v, int64_t n, bool y16) {
  const int64_t base = 4 * int64_t(group);
  if (y16 && base + 4 <= n) {
    // no memory clobber: the loads of later groups may be scheduled before it (nothing here reads y)
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(y + base), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w));
  } else {
    const float w[4] = {v.x, v.y, v.z, v.w};
    for (int e = 0; e < 4; ++e)
      if (base + e < n) atomicAdd(y + base + e, w[e]);
  }
}


// One CTA = G warpgroups of 128 threads; each warpgroup runs the tile loop on
// its own tiles with its own operand buffer, stages, mbarrier and TMEM
// columns (TCOLS each), sharing the E tables.  G is blockDim.x / 128.
// X3 (3xTF32) adds the low parts of Q after Y' in TMEM and a second (low-part) image of each
// table and a second A operand in shared memory.
template <int ND, int NQ, bool BF16, bool X3>
constexpr int tc_tcols() {
  using S = TcShape<ND, NQ, BF16>;
  return X3 ? round_up(2 * S::N1 + S::N2, 16) : round_up(S::D2_COL + S::N2, 16);
}
// CURVED (metric per quadrature point, read during the metric step): at most two warpgroups, so
// that each thread has the registers to keep a chunk's point metrics in flight.
template <int ND, int NQ, bool BF16, bool X3, bool CURVED = false>
constexpr int tc_max_groups() {
  return CURVED ? (512 / tc_tcols<ND, NQ, BF16, X3>() < 2 ? 512 / tc_tcols<ND, NQ, BF16, X3>() : 2)
                : (512 / tc_tcols<ND, NQ, BF16, X3>() < 4 ? 512 / tc_tcols<ND, NQ, BF16, X3>() : 4);
}
template <int ND, int NQ, bool BF16, bool X3, bool CURVED = false>
constexpr int tc_stages() {
  return tc_max_groups<ND, NQ, BF16, X3, CURVED>() < 4 ? 4 : 3;
}

template <int ND, int NQ, bool BF16, bool HAS_K, bool X3, bool CURVED>
__global__ void __launch_bounds__(kT * tc_max_groups<ND, NQ, BF16, X3, CURVED>(), 1)
    k_cg_apply_tc(const int64_t* __restrict__ tl_span, const int32_t* __restrict__ tl_list,
                  const uint16_t* __restrict__ tl_lidx, const float* __restrict__ metric,
                  const uint8_t* __restrict__ bimg, const float* __restrict__ u, float* __restrict__ y,
                  const float* __restrict__ kcoef, int64_t nc, int64_t ntiles, int lmax, uint32_t tmem_cols,
                  int32_t* __restrict__ status, const float* __restrict__ qmetric, int64_t ndofs, int aligned) {
  using S = TcShape<ND, NQ, BF16>;
  using St = Stage<ND, NQ, HAS_K>;
  static_assert(!(X3 && BF16), "3xTF32 splits TF32 operands");
  constexpr int KS = NQ | 1;
  constexpr int NDP = round_up(ND, 2);
  constexpr int TCOLS = tc_tcols<ND, NQ, BF16, X3>();
  constexpr int NIMG = X3 ? 2 : 1;            // high (and low) parts of the tables and of U'
  constexpr int QLO = S::N1 + S::N2;          // X3: TMEM columns of the low part of Q
  constexpr int IMG_BYTES = S::B1_BYTES + S::B2_BYTES;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int G = blockDim.x / kT;
  const int g = threadIdx.x / kT;   // warpgroup
  const int m = threadIdx.x % kT;   // row of the tile = TMEM lane
  const int warp = threadIdx.x >> 5;
  const bool u16 = aligned & 1, y16 = aligned & 2;  // u, y 16-byte aligned
  uint8_t* sB1 = smem;                        // [B1 | B2] high parts, then [B1 | B2] low parts (X3)
  uint8_t* sB2 = sB1 + S::B1_BYTES;
  uint8_t* sA1 = smem + NIMG * IMG_BYTES + size_t(g) * NIMG * S::A1_BYTES;
  uint8_t* misc = smem + NIMG * IMG_BYTES + size_t(G) * NIMG * S::A1_BYTES;  // [G][32]: mbarrier, TMEM slot
  uint64_t* bar = reinterpret_cast<uint64_t*>(misc + 32 * g);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 8);       // warpgroup 0's slot
  uint32_t* wmax = reinterpret_cast<uint32_t*>(misc + 32 * g + 16);  // per-warp maxima
  const size_t sbytes = stage_bytes<ND, NQ, HAS_K>(lmax);
  constexpr int kStages = tc_stages<ND, NQ, BF16, X3, CURVED>();
  constexpr int D = kStages - 2;  // gather distance: values of tile t + D are copied during tile t
  uint8_t* stage_base = misc + 32 * G + size_t(g) * kStages * sbytes;
  auto stage = [&](int i) { return stage_at<ND, NQ, HAS_K>(stage_base + size_t(i) * sbytes, lmax); };

  {
    const uint4* src = reinterpret_cast<const uint4*>(bimg);
    uint4* dst = reinterpret_cast<uint4*>(sB1);
    for (int i = threadIdx.x; i < NIMG * IMG_BYTES / 16; i += blockDim.x) dst[i] = src[i];
  }
  const uint32_t bar_a = smem_u32(bar);
  if (m == 0) mbar_init(bar_a);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // Prefetch ring.  During tile t the gather of tile t+D and the metadata of tile t+D+1 are issued
  // (empty groups past the last tile).  D = 2: both are awaited during tile t+1, before its GEMM 1
  // completes, so a gather has about one tile of time to arrive.  D = 1: the metadata is awaited
  // there and the gather at the end of tile t.
  const int64_t stride = int64_t(gridDim.x) * G;
  int64_t tile = int64_t(blockIdx.x) * G + g;
  int L_cur = 0, L_next = 0, L_next2 = 0;
  if (tile < ntiles)
    L_cur = issue_meta<ND, NQ, HAS_K>(stage(0), m, tile, load_span(tl_span, tile, ntiles), tl_list, tl_lidx, kcoef, nc);
  else
    cp_async_commit();
  cp_async_wait_group<0>();
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + uint32_t(g * TCOLS);
  const uint32_t lane_base = tmem + (uint32_t((warp & 3) * 32) << 16);
  const uint32_t aA1 = smem_u32(sA1), aB1 = smem_u32(sB1), aB2 = smem_u32(sB2);
  if (tile < ntiles) issue_gather<ND, NQ, HAS_K>(stage(0), m, L_cur, u, ndofs, u16);
  else cp_async_commit();
  if (tile + stride < ntiles)
    L_next = issue_meta<ND, NQ, HAS_K>(stage(1), m, tile + stride, load_span(tl_span, tile + stride, ntiles), tl_list, tl_lidx, kcoef, nc);
  else
    cp_async_commit();
  if constexpr (D == 2) {
    cp_async_wait_group<0>();
    wg_sync(g);
    if (tile + stride < ntiles) issue_gather<ND, NQ, HAS_K>(stage(1), m, L_next, u, ndofs, u16);
    else cp_async_commit();
    if (tile + 2 * stride < ntiles)
      L_next2 = issue_meta<ND, NQ, HAS_K>(stage(2), m, tile + 2 * stride, load_span(tl_span, tile + 2 * stride, ntiles), tl_list, tl_lidx, kcoef, nc);
    else
      cp_async_commit();
  } else {
    cp_async_wait_group<1>();
    wg_sync(g);
  }
  uint32_t phase = 0;
  bool failed = false;
  int b = 0;
  // software pipeline across tiles: GEMM 2 of tile t-1 runs while the rows of tile t are built,
  // GEMM 1 of tile t runs while tile t-1 is scattered and flushed
  bool have_prev = false;
  int L_prev = 0;
  uint32_t lw_prev[NDP / 2];
#pragma unroll
  for (int w = 0; w < NDP / 2; ++w) lw_prev[w] = 0u;

  // tile t-1's scatter: row m of Y' from TMEM, y_0 = -sum, fixed-point pre-reduction in shared
  // memory, then one atomic per distinct DoF.  The pre-reduction adds 32-bit integers (native
  // shared-memory atomics, no compare-and-swap retries, order-independent): every contribution of
  // the tile is scaled by 2^(24 - E), where 2^E bounds the tile's largest |contribution|; a slot
  // receives at most 128 contributions (one per cell), so no sum overflows, and the quantum
  // 2^(E - 24) is below 1.2e-7 of the largest contribution.  Tiles with a non-finite contribution
  // fall back to float atomics.
  bool fill_done = false;  // the zero-fill of y launched before this kernel (the first scatter waits)
  auto scatter = [&](const St& st, int Ls, const uint32_t* lwp) {
    if (!fill_done) {
      asm volatile("griddepcontrol.wait;" ::: "memory");
      fill_done = true;
    }
    uint32_t r[S::N2];
#pragma unroll
    for (int c = 0; c < S::N2 / 16; ++c) tmem_ld16(lane_base + S::D2_COL + 16 * c, r + 16 * c);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < S::N2 / 16; ++c) reg_fence16(r + 16 * c);
    auto pos = [&](int j) { return (lwp[j >> 1] >> (16 * (j & 1))) & 0xFFFFu; };
    float yv[ND];
    float y0 = 0.0f;
    uint32_t mx = 0u;
#pragma unroll
    for (int j = 1; j < ND; ++j) {
      yv[j] = __uint_as_float(r[j - 1]);
      y0 -= yv[j];
      mx = max(mx, __float_as_uint(fabsf(yv[j])));
    }
    yv[0] = y0;
    mx = max(mx, __float_as_uint(fabsf(y0)));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((m & 31) == 0) wmax[m >> 5] = mx;
    wg_sync(g);
    mx = max(max(wmax[0], wmax[1]), max(wmax[2], wmax[3]));
    const int E = mx ? max(int((mx >> 23) & 0xFFu) - 126, -100) : 0;  // max |y| < 2^E
    if (E <= 128) {
      const float scale = __int_as_float((127 + 24 - E) << 23);
      int* iv = reinterpret_cast<int*>(st.vals);
#pragma unroll
      for (int j = 0; j < ND; ++j) atomicAdd(iv + pos(j), __float2int_rn(yv[j] * scale));
      wg_sync(g);
      const float inv = __int_as_float((127 - 24 + E) << 23);
      const int4* i4 = reinterpret_cast<const int4*>(iv);
      for (int i = m; i < Ls; i += kT) {
        const int4 a = i4[i];
        flush_group(y, st.list[i], make_float4(float(a.x) * inv, float(a.y) * inv, float(a.z) * inv, float(a.w) * inv),
                    ndofs, y16);
      }
    } else {
#pragma unroll
      for (int j = 0; j < ND; ++j) atomicAdd(st.vals + pos(j), yv[j]);
      wg_sync(g);
      for (int i = m; i < Ls; i += kT)
        flush_group(y, st.list[i], reinterpret_cast<const float4*>(st.vals)[i], ndofs, y16);
    }
  };

  // the span of the tile whose metadata is copied next, and (affine cells) the metric of the
  // current tile, both loaded one tile ahead
  Span sp_next = load_span(tl_span, tile + (D + 1) * stride, ntiles);
  Metric met_next;
  if constexpr (!CURVED) met_next = load_metric(metric, tile, ntiles, m);
  for (; tile < ntiles; tile += stride, b = (b + 1 == kStages ? 0 : b + 1)) {
    const int bg = (b + D) % kStages;      // tile t+D: gather target
    const int bm = (b + D + 1) % kStages;  // tile t-1 (flushed), then the metadata of t+D+1
    const St cur = stage(b);
    const int64_t tg = tile + D * stride, tm = tile + (D + 1) * stride;
    // this cell's metric, consumed after GEMM 1; curved cells read one metric per point during the
    // metric step instead
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f;
    if constexpr (!CURVED) {
      m0 = met_next.v[0], m1 = met_next.v[1], m2 = met_next.v[2], m3 = met_next.v[3], m4 = met_next.v[4],
      m5 = met_next.v[5];
      met_next = load_metric(metric, tile + stride, ntiles, m);
    }
    const int L = L_cur;
    int L_new = 0;
    // 1. row m of U' from the staged values (difference form); node positions stay in registers
    uint32_t lw[NDP / 2];
#pragma unroll
    for (int w = 0; w < NDP / 2; ++w) lw[w] = cur.lidx[w * kT + m];
    {
      auto pos = [&](int j) { return (lw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu; };
      const float ue0 = cur.vals[pos(0)];
      float v1[S::K1];
#pragma unroll
      for (int j = 1; j < ND; ++j) v1[j - 1] = cur.vals[pos(j)] - ue0;
#pragma unroll
      for (int j = S::ND1; j < S::K1; ++j) v1[j] = 0.0f;
      if constexpr (X3) {
        float lo[S::K1];
#pragma unroll
        for (int j = 0; j < S::K1; ++j) {
          const float h = __uint_as_float(tf32_hi(__float_as_uint(v1[j])));
          lo[j] = v1[j] - h;
          v1[j] = h;
        }
        write_row<S::K1, false>(sA1 + S::A1_BYTES, m, lo);
      }
      write_row<S::K1, BF16>(sA1, m, v1);
    }
    fence_proxy_async();
    // GEMM 2 of tile t-1 must be complete before GEMM 1 of tile t overwrites Q in TMEM
    if (have_prev && m == 0) failed |= !mbar_wait(bar_a, phase);
    if (have_prev) phase ^= 1;
    tc_fence_before();
    failed = wg_any(g, failed);
    if (failed) break;
    tc_fence_after();
    // 2. GEMM 1 of tile t; meanwhile clear tile t's accumulator and scatter tile t-1
    if (m == 0) {
#pragma unroll
      for (int s = 0; s < S::K1 / S::KSTEP; ++s) {
        const uint64_t a_hi = smem_desc(aA1 + s * 2 * S::LBO_A, S::LBO_A, 128);
        const uint64_t b_hi = smem_desc(aB1 + s * 2 * S::LBO_B1, S::LBO_B1, 128);
        if constexpr (X3) {
          // small products first: A_lo B_hi + A_hi B_lo, then A_hi B_hi
          mma<BF16>(tmem, smem_desc(aA1 + S::A1_BYTES + s * 2 * S::LBO_A, S::LBO_A, 128), b_hi, S::idesc(S::N1),
                    s > 0);
          mma<BF16>(tmem, a_hi, smem_desc(aB1 + IMG_BYTES + s * 2 * S::LBO_B1, S::LBO_B1, 128), S::idesc(S::N1), 1);
          mma<BF16>(tmem, a_hi, b_hi, S::idesc(S::N1), 1);
        } else {
          mma<BF16>(tmem, a_hi, b_hi, S::idesc(S::N1), s > 0);
        }
      }
      mma_commit(bar_a);
    }
    for (int i = m; i < L + 1; i += kT) reinterpret_cast<float4*>(cur.vals)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (have_prev) scatter(stage(bm), L_prev, lw_prev);
    cp_async_wait_group<0>();  // this thread's share of the metadata of t+D (and, D = 2, values of t+1)
    // one thread waits for GEMM 1; the barrier also publishes the copies awaited above and the end of
    // tile t-1's flush (its stage is refilled next)
    if (m == 0) failed |= !mbar_wait(bar_a, phase);
    phase ^= 1;
    failed = wg_any(g, failed);
    if (failed) break;
    tc_fence_after();
    // gather of tile t+D, metadata of tile t+D+1
    if (tg < ntiles) issue_gather<ND, NQ, HAS_K>(stage(bg), m, D == 2 ? L_next2 : L_next, u, ndofs, u16);
    else cp_async_commit();
    if (tm < ntiles)
      L_new = issue_meta<ND, NQ, HAS_K>(stage(bm), m, tm, sp_next, tl_list, tl_lidx, kcoef, nc);
    else
      cp_async_commit();
    sp_next = load_span(tl_span, tm + stride, ntiles);
    // 3. D_e per quadrature point: G in TMEM becomes Q = (k_q) M_e g_q (w_q is folded into the table of GEMM 2)
    metric_to_q<ND, NQ, BF16, HAS_K, X3, CURVED>(lane_base, m0, m1, m2, m3, m4, m5, HAS_K ? cur.kt + m * KS : nullptr,
                                                 QLO, CURVED ? qmetric + tile * NQ * 6 * kT + m : nullptr);
    tmem_wait_st();
    tc_fence_before();
    wg_sync(g);
    // 4. GEMM 2 of tile t (A = Q in TMEM); its completion is awaited before GEMM 1 of tile t+1
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < S::K2 / S::KSTEP; ++s) {
        const uint64_t b_hi = smem_desc(aB2 + s * 2 * S::LBO_B2, S::LBO_B2, 128);
        if constexpr (X3) {
          mma_ta<BF16>(tmem + S::D2_COL, tmem + QLO + 8 * s, b_hi, S::idesc(S::N2), s > 0);
          mma_ta<BF16>(tmem + S::D2_COL, tmem + 8 * s, smem_desc(aB2 + IMG_BYTES + s * 2 * S::LBO_B2, S::LBO_B2, 128),
                       S::idesc(S::N2), 1);
          mma_ta<BF16>(tmem + S::D2_COL, tmem + 8 * s, b_hi, S::idesc(S::N2), 1);
        } else {
          mma_ta<BF16>(tmem + S::D2_COL, tmem + 8 * s, b_hi, S::idesc(S::N2), s > 0);
        }
      }
      mma_commit(bar_a);
    }
    have_prev = true;
    L_prev = L;
#pragma unroll
    for (int w = 0; w < NDP / 2; ++w) lw_prev[w] = lw[w];
    L_cur = L_next;
    if constexpr (D == 2) {
      L_next = L_next2;
      L_next2 = L_new;
    } else {
      L_next = L_new;
      cp_async_wait_group<1>();  // gather of tile t+1 (this thread's share; published by the barrier)
      wg_sync(g);
    }
  }
  // the last tile's scatter
  if (have_prev && !failed) {
    if (m == 0) failed |= !mbar_wait(bar_a, phase);
    tc_fence_before();
    failed = wg_any(g, failed);
    if (!failed) {
      tc_fence_after();
      scatter(stage(b == 0 ? kStages - 1 : b - 1), L_prev, lw_prev);
    }
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(tmem_cols));
  if (failed && m == 0) atomicOr(status, 1);
}

// ---- warp-specialised variant ----------------------------------------------------------------
// G compute warpgroups (one TMEM tile each: rows, GEMM 1, metric step, GEMM 2) and one scatter
// warpgroup that takes every finished tile off their hands: it reads Y' straight from the compute
// warpgroup's TMEM columns, pre-reduces it into that tile's stage and adds the distinct values to
// y, so the scatter no longer sits on the compute warpgroups' critical path.  Per compute
// warpgroup four mbarriers order the hand-offs, each completing once per tile:
//   g1: GEMM 1 done (compute);  g2: GEMM 2 done (compute, scatter);  rdy: tile's stage ready for
//   the scatter;  yfree: Y' read by the scatter (GEMM 2 of the next tile may overwrite it);
//   and a counter of the warpgroup's flushed tiles (their stages may be refilled).
// The scatter warpgroup visits tiles in the compute warpgroups' round-robin order; every signal is
// awaited before the next phase of the same barrier can complete, so parities never run two
// phases ahead.  Waits are bounded (about 1 s) and share an abort flag: once one gives up, every
// other wait returns at once and all warpgroups leave their loops.

template <int ND, int NQ, bool BF16>
constexpr int ws_groups() {
  return tc_max_groups<ND, NQ, BF16, false, false>();
}

// Four stages per compute warpgroup: during tile k the values of tile k+2 are gathered and the
// metadata of tile k+3 is copied into the stage of tile k-1 once the scatter has flushed it.  That
// release is a count of flushed tiles (released and acquired in shared memory), which stays valid
// however far the scatter runs ahead.
template <int ND, int NQ, bool BF16>
__global__ void __launch_bounds__(kT * (ws_groups<ND, NQ, BF16>() + 1), 1)
    k_cg_apply_tc_ws(const int64_t* __restrict__ tl_span, const int32_t* __restrict__ tl_list,
                     const uint16_t* __restrict__ tl_lidx, const float* __restrict__ metric,
                     const uint8_t* __restrict__ bimg, const float* __restrict__ u, float* __restrict__ y,
                     int64_t nc, int64_t ntiles, int lmax, uint32_t tmem_cols, int32_t* __restrict__ status,
                     int64_t ndofs, int aligned) {
  using S = TcShape<ND, NQ, BF16>;
  using St = Stage<ND, NQ, false>;
  constexpr int NDP = round_up(ND, 2);
  constexpr int TCOLS = tc_tcols<ND, NQ, BF16, false>();
  constexpr int kStages = 4;
  constexpr int IMG_BYTES = S::B1_BYTES + S::B2_BYTES;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int G = blockDim.x / kT - 1;  // compute warpgroups
  // roles: the scatter warpgroup is hardware warpgroup 0 (the lowest warp numbers, which the warp
  // schedulers favour: the scatter serves every tile and sets the pace), compute warpgroups
  // 0..G-1 are hardware warpgroups 1..G; g is the role index (G = scatter)
  const int g = threadIdx.x < kT ? G : int(threadIdx.x / kT) - 1;
  const int m = threadIdx.x % kT;
  const int warp = threadIdx.x >> 5;
  const bool u16 = aligned & 1, y16 = aligned & 2;  // u, y 16-byte aligned
  uint8_t* sB1 = smem;
  uint8_t* sB2 = sB1 + S::B1_BYTES;
  uint8_t* misc = smem + IMG_BYTES + size_t(G) * S::A1_BYTES;  // [G][64] barriers, then TMEM slot, abort, maxima
  auto bars = [&](int gg) { return smem_u32(misc + 64 * gg); };  // g1, g2, rdy, yfree, flushed (8 bytes each)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 64 * G);
  volatile int* abort = reinterpret_cast<volatile int*>(misc + 64 * G + 4);
  uint32_t* wmax = reinterpret_cast<uint32_t*>(misc + 64 * G + 16);
  const size_t sbytes = stage_bytes<ND, NQ, false>(lmax);
  uint8_t* stages = misc + 64 * G + 64;
  auto stage_of = [&](int gg, int i) {
    return stage_at<ND, NQ, false>(stages + (size_t(gg) * kStages + i) * sbytes, lmax);
  };
  const int64_t stride = int64_t(gridDim.x) * G;
  // the first three tiles' spans, in flight while the tables are copied
  const int64_t tile0 = int64_t(blockIdx.x) * G + g;
  const Span sp0 = load_span(tl_span, g < G ? tile0 : ntiles, ntiles);
  const Span sp1 = load_span(tl_span, g < G ? tile0 + stride : ntiles, ntiles);
  const Span sp2 = load_span(tl_span, g < G ? tile0 + 2 * stride : ntiles, ntiles);
  {
    const uint4* src = reinterpret_cast<const uint4*>(bimg);
    uint4* dst = reinterpret_cast<uint4*>(sB1);
    for (int i = threadIdx.x; i < IMG_BYTES / 16; i += blockDim.x) dst[i] = src[i];
  }
  if (g < G && m == 0) {
    for (int k = 0; k < 4; ++k) mbar_init(bars(g) + 8 * k);
    st_release_u32(bars(g) + 32, 0u);  // flushed tiles of this compute warpgroup
  }
  if (threadIdx.x == 0) *abort = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  bool failed = false;

  if (g < G) {
    // ---- compute warpgroup ----
    uint8_t* sA1 = smem + IMG_BYTES + size_t(g) * S::A1_BYTES;
    auto stage = [&](int i) { return stage_of(g, i); };
    const uint32_t b_g1 = bars(g), b_g2 = bars(g) + 8, b_rdy = bars(g) + 16, b_yfree = bars(g) + 24,
                   b_flushed = bars(g) + 32;
    int64_t tile = tile0;
    int L_cur = 0, L_next = 0, L_next2 = 0;
    // prologue, three dependent round trips (span, then list, then values): the metadata of tiles
    // 0 and 1, the values of tile 0 once its list is in, then the values of tile 1 and the
    // metadata of tile 2; one cp.async group each
    if (tile < ntiles) L_cur = issue_meta<ND, NQ, false>(stage(0), m, tile, sp0, tl_list, tl_lidx, nullptr, nc);
    else cp_async_commit();
    if (tile + stride < ntiles)
      L_next = issue_meta<ND, NQ, false>(stage(1), m, tile + stride, sp1, tl_list, tl_lidx, nullptr, nc);
    else
      cp_async_commit();
    cp_async_wait_group<1>();  // metadata of tile 0
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot + uint32_t(g * TCOLS);
    const uint32_t lane_base = tmem + (uint32_t((warp & 3) * 32) << 16);
    const uint32_t aA1 = smem_u32(sA1), aB1 = smem_u32(sB1), aB2 = smem_u32(sB2);
    if (tile < ntiles) issue_gather<ND, NQ, false>(stage(0), m, L_cur, u, ndofs, u16);
    else cp_async_commit();
    cp_async_wait_group<1>();  // metadata of tile 1
    wg_sync(g);
    if (tile + stride < ntiles) issue_gather<ND, NQ, false>(stage(1), m, L_next, u, ndofs, u16);
    else cp_async_commit();
    if (tile + 2 * stride < ntiles)
      L_next2 = issue_meta<ND, NQ, false>(stage(2), m, tile + 2 * stride, sp2, tl_list, tl_lidx, nullptr, nc);
    else
      cp_async_commit();
    cp_async_wait_group<2>();  // values of tile 0
    wg_sync(g);
    int b = 0;
    // the span of the tile whose metadata is copied next and the metric of the current tile, both
    // loaded one tile ahead
    Span sp_next = load_span(tl_span, tile + 3 * stride, ntiles);
    Metric met_next = load_metric(metric, tile, ntiles, m);
    for (uint32_t k = 0; tile < ntiles; tile += stride, ++k, b = (b + 1 == kStages ? 0 : b + 1)) {
      const int bg = (b + 2) % kStages, bm = (b + 3) % kStages;  // bm: held tile k + 3 - kStages
      const St cur = stage(b);
      const int64_t tg = tile + 2 * stride, tm = tile + 3 * stride;
      const float m0 = met_next.v[0], m1 = met_next.v[1], m2 = met_next.v[2], m3 = met_next.v[3],
                  m4 = met_next.v[4], m5 = met_next.v[5];
      met_next = load_metric(metric, tile + stride, ntiles, m);
      const int L = L_cur;
      int L_new = 0;
      // rows of U' (difference form)
      {
        uint32_t lw[NDP / 2];
#pragma unroll
        for (int w = 0; w < NDP / 2; ++w) lw[w] = cur.lidx[w * kT + m];
        auto pos = [&](int j) { return (lw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu; };
        const float ue0 = cur.vals[pos(0)];
        float v1[S::K1];
#pragma unroll
        for (int j = 1; j < ND; ++j) v1[j - 1] = cur.vals[pos(j)] - ue0;
#pragma unroll
        for (int j = S::ND1; j < S::K1; ++j) v1[j] = 0.0f;
        write_row<S::K1, BF16>(sA1, m, v1);
      }
      fence_proxy_async();
      // GEMM 2 of the previous tile must be complete before GEMM 1 overwrites Q
      if (k > 0 && m == 0) failed |= !mbar_wait_ab(b_g2, (k - 1) & 1, abort);
      tc_fence_before();
      failed = wg_any(g, failed);
      if (failed) break;
      tc_fence_after();
      if (m == 0) {
#pragma unroll
        for (int s = 0; s < S::K1 / S::KSTEP; ++s)
          mma<BF16>(tmem, smem_desc(aA1 + s * 2 * S::LBO_A, S::LBO_A, 128),
                    smem_desc(aB1 + s * 2 * S::LBO_B1, S::LBO_B1, 128), S::idesc(S::N1), s > 0);
        mma_commit(b_g1);
      }
      // the tile's accumulator (its values were read into the rows above)
      for (int i = m; i < L + 1; i += kT) reinterpret_cast<float4*>(cur.vals)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      cp_async_wait_group<0>();  // values of t+1, metadata of t+2 (this thread's share)
      if (m == 0) failed |= !mbar_wait_ab(b_g1, k & 1, abort);
      failed = wg_any(g, failed);
      if (failed) break;
      tc_fence_after();
      // gather of t+2; metadata of t+3 into the stage of t-1 once the scatter has flushed it
      if (tg < ntiles) issue_gather<ND, NQ, false>(stage(bg), m, L_next2, u, ndofs, u16);
      else cp_async_commit();
      if (k + 3 >= kStages) failed |= !count_wait_ab(b_flushed, k + 4 - kStages, abort);
      if (tm < ntiles)
        L_new = issue_meta<ND, NQ, false>(stage(bm), m, tm, sp_next, tl_list, tl_lidx, nullptr, nc);
      else
        cp_async_commit();
      sp_next = load_span(tl_span, tm + stride, ntiles);
      // TF32 keeps one chunk live at a time (the warp-specialised kernel runs at 128 registers)
      metric_to_q<ND, NQ, BF16, false, false, false, !BF16>(lane_base, m0, m1, m2, m3, m4, m5, nullptr);
      tmem_wait_st();
      tc_fence_before();
      wg_sync(g);
      if (m == 0) {
        // the scatter has read the previous tile's Y' (GEMM 2 overwrites it); then hand this tile over
        if (k > 0) failed |= !mbar_wait_ab(b_yfree, (k - 1) & 1, abort);
        mbar_arrive(b_rdy);
        tc_fence_after();
#pragma unroll
        for (int s = 0; s < S::K2 / S::KSTEP; ++s)
          mma_ta<BF16>(tmem + S::D2_COL, tmem + 8 * s, smem_desc(aB2 + s * 2 * S::LBO_B2, S::LBO_B2, 128),
                       S::idesc(S::N2), s > 0);
        mma_commit(b_g2);
      }
      L_cur = L_next;
      L_next = L_next2;
      L_next2 = L_new;
    }
    cp_async_wait_all();
    failed = wg_any(g, failed);
  } else {
    // ---- scatter warpgroup ----
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the kernel may start while the zero-fill of y (launched before it) still runs: the scatter
    // is the only part that touches y
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint32_t tbase = *tslot + (uint32_t((warp & 3) * 32) << 16);
    for (uint32_t k = 0; !failed && int64_t(blockIdx.x) * G + int64_t(k) * stride < ntiles; ++k) {
      for (int gg = 0; gg < G; ++gg) {
        const int64_t t = int64_t(blockIdx.x) * G + gg + int64_t(k) * stride;
        if (t >= ntiles) break;
        const uint32_t bb = bars(gg);
        bool f = !mbar_wait_ab(bb + 16, k & 1, abort);  // stage ready
        f = f || !mbar_wait_ab(bb + 8, k & 1, abort);   // GEMM 2 done
        failed = wg_any(G, f);
        if (failed) break;
        tc_fence_after();
        uint32_t r[S::N2];
#pragma unroll
        for (int c = 0; c < S::N2 / 16; ++c) tmem_ld16(tbase + gg * TCOLS + S::D2_COL + 16 * c, r + 16 * c);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < S::N2 / 16; ++c) reg_fence16(r + 16 * c);
        tc_fence_before();
        const St st = stage_of(gg, int(k % kStages));
        uint32_t lw[NDP / 2];
#pragma unroll
        for (int w = 0; w < NDP / 2; ++w) lw[w] = st.lidx[w * kT + m];
        auto pos = [&](int j) { return (lw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu; };
        const int Ls = int(__ldg(tl_span + 2 * t + 1));
        float yv[ND];
        float y0 = 0.0f;
        uint32_t mx = 0u;
#pragma unroll
        for (int j = 1; j < ND; ++j) {
          yv[j] = __uint_as_float(r[j - 1]);
          y0 -= yv[j];
          mx = max(mx, __float_as_uint(fabsf(yv[j])));
        }
        yv[0] = y0;
        mx = max(mx, __float_as_uint(fabsf(y0)));
        mx = __reduce_max_sync(0xffffffffu, mx);
        if ((m & 31) == 0) wmax[m >> 5] = mx;
        wg_sync(G);
        if (m == 0) mbar_arrive(bb + 24);  // Y' read: GEMM 2 of the next tile may overwrite it
        mx = max(max(wmax[0], wmax[1]), max(wmax[2], wmax[3]));
        const int E = mx ? max(int((mx >> 23) & 0xFFu) - 126, -100) : 0;
        if (E <= 128) {
          const float scale = __int_as_float((127 + 24 - E) << 23);
          int* iv = reinterpret_cast<int*>(st.vals);
#pragma unroll
          for (int j = 0; j < ND; ++j) atomicAdd(iv + pos(j), __float2int_rn(yv[j] * scale));
          wg_sync(G);
          const float inv = __int_as_float((127 - 24 + E) << 23);
          const int4* i4 = reinterpret_cast<const int4*>(iv);
          // two groups per thread and round, both loaded before either is added
          for (int i = m; i < Ls; i += 2 * kT) {
            const bool two = i + kT < Ls;
            const int4 a = i4[i];
            const int32_t ga = st.list[i];
            const int4 c = two ? i4[i + kT] : make_int4(0, 0, 0, 0);
            const int32_t gc = two ? st.list[i + kT] : 0;
            flush_group(y, ga, make_float4(float(a.x) * inv, float(a.y) * inv, float(a.z) * inv, float(a.w) * inv),
                        ndofs, y16);
            if (two)
              flush_group(y, gc, make_float4(float(c.x) * inv, float(c.y) * inv, float(c.z) * inv, float(c.w) * inv),
                          ndofs, y16);
          }
        } else {
#pragma unroll
          for (int j = 0; j < ND; ++j) atomicAdd(st.vals + pos(j), yv[j]);
          wg_sync(G);
          for (int i = m; i < Ls; i += kT)
            flush_group(y, st.list[i], reinterpret_cast<const float4*>(st.vals)[i], ndofs, y16);
        }
        wg_sync(G);  // the flush of this stage is complete (and wmax may be reused)
        if (m == 0) st_release_u32(bb + 32, k + 1);  // tiles 0..k of this warpgroup are flushed
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(tmem_cols));
  if (failed && m == 0) atomicOr(status, 1);
}

// TF32 value of v as the image stores it (round to nearest, ties away from zero)
double tf32_value(double v) {
  float f = float(v);
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  bits = (bits + 0x1000u) & 0xFFFFE000u;
  std::memcpy(&f, &bits, 4);
  return double(f);
}

// Operand images of the two tables; X3: the TF32 high parts, then the low parts (table - high part)
template <int ND, int NQ, bool BF16, bool X3>
std::vector<uint8_t> b_image(const RefTables& t) {
  using S = TcShape<ND, NQ, BF16>;
  constexpr size_t IMG = S::B1_BYTES + S::B2_BYTES;
  std::vector<uint8_t> img((X3 ? 2 : 1) * IMG, 0);
  auto off = [](int r, int k, int lbo) {
    return size_t((k / S::KC) * lbo + (r / 8) * 128 + (r % 8) * 16 + (k % S::KC) * S::ES);
  };
  // B1 = E' as [N1 rows = grad_col(q, k)][K1 = j-1]; B2 = (w E')^T as [N2 rows = j-1][K2 = grad_col(q, k)]
  // (the quadrature weight w_q is folded into the integration table)
  for (int q = 0; q < NQ; ++q)
    for (int k = 0; k < 3; ++k)
      for (int j = 1; j < ND; ++j) {
        const double e = t.E[(size_t(q) * 3 + k) * ND + j];
        const double ew = e * t.wq[q];
        const int n = grad_col(q, k);
        put_elem<BF16>(img, off(n, j - 1, S::LBO_B1), e);
        put_elem<BF16>(img, S::B1_BYTES + off(j - 1, n, S::LBO_B2), ew);
        if (X3) {
          put_elem<false>(img, IMG + off(n, j - 1, S::LBO_B1), e - tf32_value(e));
          put_elem<false>(img, IMG + S::B1_BYTES + off(j - 1, n, S::LBO_B2), ew - tf32_value(ew));
        }
      }
  return img;
}

template <int ND, int NQ, bool BF16, bool HAS_K, bool X3, bool CURVED>
size_t tc_smem(int lmax, int G) {
  using S = TcShape<ND, NQ, BF16>;
  constexpr int NIMG = X3 ? 2 : 1;
  return size_t(NIMG) * (S::B1_BYTES + S::B2_BYTES) +
         size_t(G) * (NIMG * S::A1_BYTES + 32 +
                      tc_stages<ND, NQ, BF16, X3, CURVED>() * stage_bytes<ND, NQ, HAS_K>(lmax));
}

template <int ND, int NQ, bool BF16, bool X3>
int upload_image(Ctx& c, void** dst) {
  const std::vector<uint8_t> img = b_image<ND, NQ, BF16, X3>(c.tab);
  void* p = nullptr;
  TETMF_CK(cudaMalloc(&p, img.size()));
  c.allocations.push_back(p);
  TETMF_CK(cudaMemcpy(p, img.data(), img.size(), cudaMemcpyHostToDevice));
  *dst = p;
  return FEM_OK;
}

template <int ND, int NQ>
int prepare(Ctx& c) {
  if (int s = upload_image<ND, NQ, false, false>(c, &c.d_tc_tf32)) return s;
  if (int s = upload_image<ND, NQ, false, true>(c, &c.d_tc_tf32x3)) return s;
  return upload_image<ND, NQ, true, false>(c, &c.d_tc_bf16);
}

// bit 0: u is 16-byte aligned, bit 1: y is (the kernels then move whole groups of 4 values)
int alignment_flags(const float* u, const float* y) {
  return ((reinterpret_cast<uintptr_t>(u) & 15) == 0 ? 1 : 0) | ((reinterpret_cast<uintptr_t>(y) & 15) == 0 ? 2 : 0);
}

template <int ND, int NQ, bool BF16, bool HAS_K, bool X3, bool CURVED>
int launch_g(Ctx& c, const float* u, float* y, const float* k, cudaStream_t st) {
  constexpr int TCOLS = tc_tcols<ND, NQ, BF16, X3>();
  const int lmax = round_up(c.tl_max, 4);
  auto kern = k_cg_apply_tc<ND, NQ, BF16, HAS_K, X3, CURVED>;
  int dev = 0, smem_max = 0;
  TETMF_CK(cudaGetDevice(&dev));
  TETMF_CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // warpgroups per CTA: as many tiles in flight per SM as TMEM (512 columns) and shared memory allow
  int G = tc_max_groups<ND, NQ, BF16, X3, CURVED>();
  while (G > 1 && tc_smem<ND, NQ, BF16, HAS_K, X3, CURVED>(lmax, G) > size_t(smem_max)) --G;
  const size_t sm = tc_smem<ND, NQ, BF16, HAS_K, X3, CURVED>(lmax, G);
  if (G < 1 || sm > size_t(smem_max)) {
    set_error("tensor-core kernel does not fit on an SM (%zu bytes of shared memory)", sm);
    return FEM_EUNSUPPORTED;
  }
  if (int e = allow_smem(kern, sm)) return e;
  const uint32_t cols = uint32_t(pow2_cols(G * TCOLS));
  int64_t grid = (c.ntiles + G - 1) / G;
  if (grid > sm_count()) grid = sm_count();
  const void* img = X3 ? c.d_tc_tf32x3 : BF16 ? c.d_tc_bf16 : c.d_tc_tf32;
  // may start while the zero-fill before it runs (the first scatter waits for it)
  TETMF_CK(launch_early(kern, dim3(unsigned(grid)), dim3(unsigned(G * kT)), sm, st, c.d_tl_span, c.d_tl_list,
                        c.d_tl_lidx, c.d_metric32, static_cast<const uint8_t*>(img), u, y, k, c.nc, c.ntiles, lmax, cols,
                        c.d_status, c.d_qmetric32, c.ndofs, alignment_flags(u, y)));
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

template <int ND, int NQ, bool BF16>
int launch_ws(Ctx& c, const float* u, float* y, cudaStream_t st) {
  using S = TcShape<ND, NQ, BF16>;
  constexpr int G = ws_groups<ND, NQ, BF16>();
  const int lmax = round_up(c.tl_max, 4);
  const size_t sm = size_t(S::B1_BYTES) + S::B2_BYTES + size_t(G) * S::A1_BYTES + 64 * G + 64 +
                    size_t(G) * 4 * stage_bytes<ND, NQ, false>(lmax);
  int dev = 0, smem_max = 0;
  TETMF_CK(cudaGetDevice(&dev));
  TETMF_CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (sm > size_t(smem_max)) return launch_g<ND, NQ, BF16, false, false, false>(c, u, y, nullptr, st);
  auto kern = k_cg_apply_tc_ws<ND, NQ, BF16>;
  if (int e = allow_smem(kern, sm)) return e;
  const uint32_t cols = uint32_t(pow2_cols(G * tc_tcols<ND, NQ, BF16, false>()));
  int64_t grid = (c.ntiles + G - 1) / G;
  if (grid > sm_count()) grid = sm_count();
  // may start while the zero-fill before it runs (the kernel waits for it before touching y)
  TETMF_CK(launch_early(kern, dim3(unsigned(grid)), dim3(unsigned((G + 1) * kT)), sm, st, c.d_tl_span, c.d_tl_list,
                        c.d_tl_lidx, c.d_metric32, static_cast<const uint8_t*>(BF16 ? c.d_tc_bf16 : c.d_tc_tf32), u, y,
                        c.nc, c.ntiles, lmax, cols, c.d_status, c.ndofs, alignment_flags(u, y)));
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

template <int ND, int NQ, bool BF16, bool X3>
int launch(Ctx& c, const float* u, float* y, const float* k, cudaStream_t st) {
  if (int e = init_rows<float>(y, u, c.d_mask, c.ndofs, 0.0f, st)) return e;
  if constexpr (!X3 && ws_groups<ND, NQ, BF16>() <= 3) {
    // where TMEM leaves room for at most three tiles per SM: compute warpgroups plus one warpgroup
    // that moves the data
    if (!k) return launch_ws<ND, NQ, BF16>(c, u, y, st);
  }
  return k ? launch_g<ND, NQ, BF16, true, X3, false>(c, u, y, k, st)
           : launch_g<ND, NQ, BF16, false, X3, false>(c, u, y, k, st);
}

template <int ND, int NQ>
int launch_prec(Ctx& c, int prec, const float* u, float* y, const float* k, cudaStream_t st) {
  if (c.curved) {
    // curved cells: TF32 / BF16 without a coefficient
    if (k || (prec != FEM_TF32 && prec != FEM_BF16)) {
      set_error("curved cells on the tensor cores: FEM_TF32 or FEM_BF16 without a coefficient");
      return FEM_EUNSUPPORTED;
    }
    if (int e = init_rows<float>(y, u, c.d_mask, c.ndofs, 0.0f, st)) return e;
    return prec == FEM_BF16 ? launch_g<ND, NQ, true, false, false, true>(c, u, y, k, st)
                            : launch_g<ND, NQ, false, false, false, true>(c, u, y, k, st);
  }
  if (prec == FEM_BF16) return launch<ND, NQ, true, false>(c, u, y, k, st);
  if (prec == FEM_TF32X3) {
    if constexpr (ND > 20) {
      // p = 4: the high and low images of both tables (155 KB) leave no room for the tile stages
      set_error("FEM_TF32X3 is offered for degrees 1 to 3");
      return FEM_EUNSUPPORTED;
    } else {
      return launch<ND, NQ, false, true>(c, u, y, k, st);
    }
  }
  return launch<ND, NQ, false, false>(c, u, y, k, st);
}

}  // namespace

int tc_prepare(Ctx& c) { TETMF_DISPATCH_SPACE(c.p, c.nq, (prepare<ND, NQ>(c))) }

int cg_apply_tc(Ctx& c, int prec, const void* u, void* y, const void* k, void* stream) {
  cudaStream_t st = as_stream(stream);
  const float* uf = static_cast<const float*>(u);
  float* yf = static_cast<float*>(y);
  const float* kf = static_cast<const float*>(k);
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_prec<ND, NQ>(c, prec, uf, yf, kf, st)))
}

}  // namespace tetmf
