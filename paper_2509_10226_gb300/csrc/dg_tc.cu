// Discontinuous Galerkin (SIPG, Eq. 2 / Eq. 5) apply with the interpolation
// products on the tcgen05 tensor cores (TF32 or BF16 operands, FP32 accumulate).
//
// Cell loop (k_dg_cell_tc): the CG contraction of Eq. 3 on contiguous per-cell
// DoFs, 128 cells per tile, difference form, Q in TMEM; y is written once per
// cell (no atomics).
//
// Face loop (k_dg_face_tc): faces in tiles of 128, in the Morton order of their
// minus cells (padded with faces of zero weight).  Each side's cell is relabelled
// so that the face is its local face 0 with the face's vertices in increasing
// global order: both sides then place the face points alike, and one evaluation
// and one integration table serve every face (faces of equal orientation can
// share their interpolation matrices, Sec. 3.1; here every face is brought to
// one orientation).  The relabelling only permutes a cell's DoFs (one of 24
// permutations).  Per tile:
//   1. rows of U- and U+ (both sides' DoFs in relabelled order, shifted by the
//      minus side's first DoF so that rounded tables keep jumps of smooth fields
//      small: jumps and gradients are unchanged by a common shift);
//   2. two GEMMs evaluate value and reference gradient at the face points:
//      D = U . T^T with T = [phi; d phi / d xhat] (4 nqf x nd);
//   3. per face and point the SIPG flux in FP32: jump, average normal
//      derivative (a . grad_hat with a = J'^-1 n in each relabelled frame),
//      penalty; the coefficients of the test functions (value, and a *
//      coefficient of the normal derivative) overwrite D in TMEM;
//   4. two GEMMs integrate back, Y = Q . (w T) (weights folded in the table);
//   5. both rows, back in the cells' own DoF order, are added to y with vector
//      reductions.
// The rows of U live in TMEM (the A operand of the evaluation GEMMs), and the
// DoF values and face data of the next tiles are copied ahead (cp.async).
// Boundary faces take the mirror state of the weak Dirichlet condition (u+ = -u-, equal normal
// derivatives) and go through the same tiles: their plus row is the negated minus row, with
// a+ = -a-, and only their minus side is added to y.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace tetmf {
namespace {

constexpr int kT = kTile;

template <int ND, int NQF, bool BF16>
struct FaceShape {
  static constexpr int ES = BF16 ? 2 : 4;
  static constexpr int KC = 16 / ES;
  static constexpr int KSTEP = 2 * KC;
  static constexpr int NE = round_up(4 * NQF, 16);      // evaluation GEMM N: (value, 3 gradients) per point
  static constexpr int KE = round_up(ND, KSTEP);        // evaluation GEMM K
  static constexpr int KI = round_up(4 * NQF, KSTEP);   // integration GEMM K
  static constexpr int NI = round_up(ND, 16);           // integration GEMM N
  static constexpr int TCOLS = round_up(2 * NE + 2 * NI, 16);
  static constexpr int GMAX = 512 / TCOLS < 4 ? 512 / TCOLS : 4;
  static constexpr int LBO_E = (NE / 8) * 128;
  static constexpr int LBO_I = (NI / 8) * 128;
  static constexpr int E_BYTES = NE * KE * ES;
  static constexpr int I_BYTES = NI * KI * ES;
  static constexpr uint32_t fmt = BF16 ? 1u : 2u;
  __host__ __device__ static constexpr uint32_t idesc(int n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kT >> 4) << 24);
  }
  static_assert(KI <= NE, "coefficients must fit in the evaluation columns");
};

// Operand images of local face 0 of the reference cell (every face is seen as local face 0 of
// both relabelled cells, points in the same order): the evaluation table, then the integration
// table (quadrature weights folded in).
template <int ND, int NQF, bool BF16>
std::vector<uint8_t> face_images(const RefTables& t) {
  using S = FaceShape<ND, NQF, BF16>;
  std::vector<uint8_t> img(size_t(S::E_BYTES) + size_t(S::I_BYTES), 0);
  auto off = [](int r, int k, int lbo) {
    return size_t((k / S::KC) * lbo + (r / 8) * 128 + (r % 8) * 16 + (k % S::KC) * S::ES);
  };
  // table entry: c = 0 value, c = 1..3 reference gradient, at point q of local face 0
  auto entry = [&](int q, int c, int j) {
    return c == 0 ? t.Vf[size_t(q) * ND + j] : t.Ef[(size_t(q) * 3 + (c - 1)) * ND + j];
  };
  std::vector<uint8_t> e(S::E_BYTES, 0), in(S::I_BYTES, 0);
  for (int q = 0; q < NQF; ++q)
    for (int c = 0; c < 4; ++c)
      for (int j = 0; j < ND; ++j) {
        const double v = entry(q, c, j);
        put_elem<BF16>(e, off(4 * q + c, j, S::LBO_E), v);
        put_elem<BF16>(in, off(j, 4 * q + c, S::LBO_I), v * t.wqf[q]);
      }
  std::memcpy(img.data(), e.data(), e.size());
  std::memcpy(img.data() + S::E_BYTES, in.data(), in.size());
  return img;
}

template <int ND, int NQF>
int prepare_images(Ctx& c) {
  for (int b = 0; b < 2; ++b) {
    const std::vector<uint8_t> img = b ? face_images<ND, NQF, true>(c.tab) : face_images<ND, NQF, false>(c.tab);
    void* p = nullptr;
    TETMF_CK(cudaMalloc(&p, img.size()));
    c.allocations.push_back(p);
    TETMF_CK(cudaMemcpy(p, img.data(), img.size(), cudaMemcpyHostToDevice));
    (b ? c.d_dg_img_bf16 : c.d_dg_img_tf32) = p;
  }
  return FEM_OK;
}

// ---- cell loop ------------------------------------------------------------
// Eq. 3 on contiguous per-cell DoFs (one offset per cell): 128 cells per tile, the tile's
// 128 x ND block of u arrives in one coalesced copy (cp.async, 16-byte pieces) and y leaves the
// same way, written once (the face kernels then add to it).  The GEMMs and the metric step are
// the CG ones (difference form, E tables of the CG tensor-core path).
template <int ND, int NQ, bool BF16>
constexpr int cell_tcols() {
  return round_up(TcShape<ND, NQ, BF16>::D2_COL + TcShape<ND, NQ, BF16>::N2, 16);
}
template <int ND, int NQ, bool BF16>
constexpr int cell_gmax() {
  return 512 / cell_tcols<ND, NQ, BF16>() < 4 ? 512 / cell_tcols<ND, NQ, BF16>() : 4;
}
template <int ND, int NQ, bool BF16>
constexpr size_t cell_smem(int G) {
  using S = TcShape<ND, NQ, BF16>;
  return size_t(S::B1_BYTES) + S::B2_BYTES + size_t(G) * (32 + S::A1_BYTES + 2 * size_t(kT) * ND * 4);
}

// copy a tile's block of n floats (16-byte aligned source) into shared memory
__device__ inline void issue_block(float* dst, const float* __restrict__ src, int n, int m) {
  const int n4 = n / 4;
  for (int i = m; i < n4; i += kT) cp_async16(dst + 4 * i, src + 4 * i);
  for (int i = 4 * n4 + m; i < n; i += kT) cp_async4(dst + i, src + i);
  cp_async_commit();
}

template <int ND, int NQ, bool BF16>
__global__ void __launch_bounds__(kT * cell_gmax<ND, NQ, BF16>(), 1)
    k_dg_cell_tc(const float* __restrict__ metric, const uint8_t* __restrict__ bimg, const float* __restrict__ u,
                 float* __restrict__ y, int64_t nc, int64_t ntiles, uint32_t tmem_cols, int32_t* __restrict__ status) {
  using S = TcShape<ND, NQ, BF16>;
  constexpr int TCOLS = cell_tcols<ND, NQ, BF16>();
  extern __shared__ __align__(1024) uint8_t smem[];
  // the face kernel launched after this one may start now; it waits for this kernel before it adds
  // to y
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int G = blockDim.x / kT;
  const int g = threadIdx.x / kT;
  const int m = threadIdx.x % kT;
  const int warp = threadIdx.x >> 5;
  uint8_t* misc = smem;  // [G][32]: mbarrier, TMEM slot (warpgroup 0)
  uint8_t* sB1 = smem + 32 * G;
  uint8_t* sB2 = sB1 + S::B1_BYTES;
  uint8_t* own = sB2 + S::B2_BYTES + size_t(g) * (S::A1_BYTES + 2 * size_t(kT) * ND * 4);
  uint8_t* sA1 = own;
  float* const stg0 = reinterpret_cast<float*>(own + S::A1_BYTES);  // two stages of 128 x ND values
  auto stg = [&](int i) { return stg0 + i * (kT * ND); };
  uint64_t* bar = reinterpret_cast<uint64_t*>(misc + 32 * g);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 8);
  {
    const uint4* src = reinterpret_cast<const uint4*>(bimg);
    uint4* dst = reinterpret_cast<uint4*>(sB1);
    for (int i = threadIdx.x; i < (S::B1_BYTES + S::B2_BYTES) / 16; i += blockDim.x) dst[i] = src[i];
  }
  const uint32_t bar_a = smem_u32(bar);
  if (m == 0) mbar_init(bar_a);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const int64_t stride = int64_t(gridDim.x) * G;
  int64_t tile = int64_t(blockIdx.x) * G + g;
  auto ncell_of = [&](int64_t t) { return int(nc - t * kT < kT ? nc - t * kT : kT); };
  if (tile < ntiles) issue_block(stg(0), u + tile * kT * ND, ncell_of(tile) * ND, m);
  else cp_async_commit();
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + uint32_t(g * TCOLS);
  const uint32_t lane_base = tmem + (uint32_t((warp & 3) * 32) << 16);
  const uint32_t aA1 = smem_u32(sA1), aB1 = smem_u32(sB1), aB2 = smem_u32(sB2);
  uint32_t phase = 0;
  bool failed = false;
  for (int b = 0; tile < ntiles; tile += stride, b ^= 1) {
    const int64_t next = tile + stride;
    if (next < ntiles) issue_block(stg(b ^ 1), u + next * kT * ND, ncell_of(next) * ND, m);
    else cp_async_commit();
    const int ncell = ncell_of(tile);
    float* cur = stg(b);
    cp_async_wait_group<1>();
    wg_sync(g);
    // 1. row m of U' (difference form); rows past the last cell are zero
    {
      float v1[S::K1];
      const float ue0 = m < ncell ? cur[m * ND] : 0.0f;
#pragma unroll
      for (int j = 1; j < ND; ++j) v1[j - 1] = m < ncell ? cur[m * ND + j] - ue0 : 0.0f;
#pragma unroll
      for (int j = S::ND1; j < S::K1; ++j) v1[j] = 0.0f;
      write_row<S::K1, BF16>(sA1, m, v1);
    }
    fence_proxy_async();
    tc_fence_before();
    wg_sync(g);
    // 2. GEMM 1
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < S::K1 / S::KSTEP; ++s)
        mma<BF16>(tmem, smem_desc(aA1 + s * 2 * S::LBO_A, S::LBO_A, 128),
                  smem_desc(aB1 + s * 2 * S::LBO_B1, S::LBO_B1, 128), S::idesc(S::N1), s > 0);
      mma_commit(bar_a);
    }
    const float* mp = metric + tile * 6 * kT + m;
    const float m0 = __ldg(mp), m1 = __ldg(mp + kT), m2 = __ldg(mp + 2 * kT), m3 = __ldg(mp + 3 * kT),
                m4 = __ldg(mp + 4 * kT), m5 = __ldg(mp + 5 * kT);
    if (m == 0) failed |= !mbar_wait(bar_a, phase);
    phase ^= 1;
    failed = wg_any(g, failed);
    if (failed) break;
    tc_fence_after();
    // 3. D_e per quadrature point
    metric_to_q<ND, NQ, BF16, false>(lane_base, m0, m1, m2, m3, m4, m5, nullptr);
    tmem_wait_st();
    tc_fence_before();
    wg_sync(g);
    // 4. GEMM 2 (A = Q in TMEM)
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < S::K2 / S::KSTEP; ++s)
        mma_ta<BF16>(tmem + S::D2_COL, tmem + 8 * s, smem_desc(aB2 + s * 2 * S::LBO_B2, S::LBO_B2, 128),
                     S::idesc(S::N2), s > 0);
      mma_commit(bar_a);
      failed |= !mbar_wait(bar_a, phase);
    }
    phase ^= 1;
    failed = wg_any(g, failed);
    if (failed) break;
    tc_fence_after();
    // 5. row m of Y' from TMEM, y_0 = -sum, staged and written out coalesced
    {
      uint32_t r[S::N2];
#pragma unroll
      for (int c = 0; c < S::N2 / 16; ++c) tmem_ld16(lane_base + S::D2_COL + 16 * c, r + 16 * c);
      tmem_wait_ld();
#pragma unroll
      for (int c = 0; c < S::N2 / 16; ++c) reg_fence16(r + 16 * c);
      if (m < ncell) {
        float y0 = 0.0f;
#pragma unroll
        for (int j = 1; j < ND; ++j) {
          const float v = __uint_as_float(r[j - 1]);
          cur[m * ND + j] = v;
          y0 -= v;
        }
        cur[m * ND] = y0;
      }
    }
    tc_fence_before();
    wg_sync(g);
    {
      float* dst = y + tile * kT * ND;
      const int n = ncell * ND, n4 = n / 4;
      for (int i = m; i < n4; i += kT) reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(cur)[i];
      for (int i = 4 * n4 + m; i < n; i += kT) dst[i] = cur[i];
    }
    wg_sync(g);  // the stage is refilled by the prefetch of the next iteration
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(tmem_cols));
  if (failed && m == 0) atomicOr(status, 1);
}

// ---- interior faces ---------------------------------------------------------
constexpr int kMetaWords = 11 * kTile;  // one slot of face data (see issue_face_meta)
constexpr int32_t kMirrorFace = 1 << 16;  // relabelling word: a boundary face (mirror state on its plus side)

// per warpgroup: the DoF values of both sides (one slot), their results on the way back to y
// (the rows in the cells' own DoF order) and the face data (two slots); per CTA: the two tables and
// the DoF permutations of the 24 relabellings
template <int ND, int NQF, bool BF16>
constexpr size_t face_wg_bytes() {
  return 2 * 2 * size_t(kT) * ND * 4 + 2 * size_t(kMetaWords) * 4;
}
template <int ND, int NQF, bool BF16>
constexpr size_t face_cta_bytes() {
  using S = FaceShape<ND, NQF, BF16>;
  return 128 + size_t(S::E_BYTES) + size_t(S::I_BYTES) + size_t(24) * round_up(ND, 16);
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// face data of tile t into a slot [11][128]: cells of both sides, the relabelling word, then
// a- a+ 2|F| tau
__device__ __forceinline__ void issue_face_meta(uint32_t* slot, const int32_t* __restrict__ tcell,
                                                const int32_t* __restrict__ tperm, const float* __restrict__ tgeo,
                                                int64_t t, int m) {
  for (int i = m; i < 2 * kT / 4; i += kT) cp_async16(slot + 4 * i, tcell + t * 2 * kT + 4 * i);
  for (int i = m; i < kT / 4; i += kT) cp_async16(slot + 2 * kT + 4 * i, tperm + t * kT + 4 * i);
  for (int i = m; i < 8 * kT / 4; i += kT) cp_async16(slot + 3 * kT + 4 * i, tgeo + t * 8 * kT + 4 * i);
}

// the DoF permutation of a relabelling: PROW bytes per row in shared memory (old local DoF of each
// new local DoF), held as 32-bit words; perm_at(w, j) is the old DoF of new DoF j
template <int ND>
constexpr int perm_row_bytes() {
  return round_up(ND, 16);
}
template <int ND>
__device__ __forceinline__ void load_perm(const int8_t* sP, uint32_t id, uint32_t* w) {
  const uint4* r = reinterpret_cast<const uint4*>(sP + id * perm_row_bytes<ND>());
#pragma unroll
  for (int q = 0; q < perm_row_bytes<ND>() / 16; ++q) {
    const uint4 v = r[q];
    w[4 * q] = v.x, w[4 * q + 1] = v.y, w[4 * q + 2] = v.z, w[4 * q + 3] = v.w;
  }
}
__device__ __forceinline__ int perm_at(const uint32_t* w, int j) { return int((w[j >> 2] >> (8 * (j & 3))) & 0xFFu); }

// this thread's rows of the tile: the DoF values of its face's two cells, in the cells' own order
template <int ND>
__device__ __forceinline__ void issue_face_u(float* su, const float* __restrict__ u, int64_t cm, int64_t cp, int m) {
  float* dm = su + m * ND;
  float* dp = su + (kT + m) * ND;
  const float* a = u + cm * ND;
  const float* b = u + cp * ND;
  if constexpr (ND % 4 == 0) {
#pragma unroll
    for (int j = 0; j < ND; j += 4) cp_async16(dm + j, a + j), cp_async16(dp + j, b + j);
  } else if constexpr (ND % 2 == 0) {
#pragma unroll
    for (int j = 0; j < ND; j += 2) cp_async8(dm + j, a + j), cp_async8(dp + j, b + j);
  } else {
#pragma unroll
    for (int j = 0; j < ND; ++j) cp_async4(dm + j, a + j), cp_async4(dp + j, b + j);
  }
}

// one staged row of ND values (64-bit shared loads for even ND: rows 40 bytes apart then fill
// the two wavefronts of a warp's request without bank conflicts)
template <int ND>
__device__ __forceinline__ void load_row(const float* r, float* v) {
  if constexpr (ND % 2 == 0) {
#pragma unroll
    for (int j = 0; j < ND / 2; ++j) {
      const float2 t = reinterpret_cast<const float2*>(r)[j];
      v[2 * j] = t.x, v[2 * j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < ND; ++j) v[j] = r[j];
  }
}

__device__ __forceinline__ void red_v4(float* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(__uint_as_float(a)), "f"(__uint_as_float(b)),
               "f"(__uint_as_float(c)), "f"(__uint_as_float(d))
               : "memory");
}
__device__ __forceinline__ void red_v2(float* p, uint32_t a, uint32_t b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(__uint_as_float(a)), "f"(__uint_as_float(b))
               : "memory");
}

// y[0..ND) += v with vector reductions (no return value).  Rows of ND = 2 mod 4 values start on
// an 8-byte boundary: 16-byte pieces where the row is 16-byte aligned, else one 8-byte piece
// first; the operands are selected without divergence.
template <int ND>
__device__ __forceinline__ void red_cell(float* p, const uint32_t* v) {
  if constexpr (ND % 4 == 0) {
#pragma unroll
    for (int j = 0; j < ND / 4; ++j) red_v4(p + 4 * j, v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  } else if constexpr (ND % 2 == 0) {
    const bool a16 = (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
    const int o4 = a16 ? 0 : 2;
#pragma unroll
    for (int j = 0; j < ND / 4; ++j)
      red_v4(p + o4 + 4 * j, a16 ? v[4 * j] : v[4 * j + 2], a16 ? v[4 * j + 1] : v[4 * j + 3],
             a16 ? v[4 * j + 2] : v[4 * j + 4], a16 ? v[4 * j + 3] : v[4 * j + 5]);
    red_v2(p + (a16 ? ND - 2 : 0), a16 ? v[ND - 2] : v[0], a16 ? v[ND - 1] : v[1]);
  } else {
#pragma unroll
    for (int j = 0; j < ND; ++j) atomicAdd(p + j, __uint_as_float(v[j]));
  }
}

// one row of U (values minus the shift, zero past ND) as TMEM words: FP32 bits (TF32 operand)
// or packed BF16 pairs
template <int ND, int KE, bool BF16>
__device__ __forceinline__ void pack_row(const float* v, float sh, uint32_t* w) {
  if constexpr (BF16) {
#pragma unroll
    for (int j = 0; j < KE / 2; ++j)
      w[j] = pack_bf16(2 * j < ND ? v[2 * j] - sh : 0.0f, 2 * j + 1 < ND ? v[2 * j + 1] - sh : 0.0f);
  } else {
#pragma unroll
    for (int j = 0; j < KE; ++j) w[j] = __float_as_uint(j < ND ? v[j] - sh : 0.0f);
  }
}

// W consecutive TMEM columns of this thread's lane (W a multiple of 8)
template <int W>
__device__ __forceinline__ void tmem_st_row(uint32_t taddr, const uint32_t* w) {
#pragma unroll
  for (int c = 0; c + 16 <= W; c += 16) tmem_st16(taddr + c, w + c);
  if constexpr (W % 16 == 8) tmem_st8(taddr + (W - 8), w + (W - 8));
}

// One CTA = G warpgroups sharing the two face-0 tables; warpgroup w of the grid takes a contiguous
// run of tiles (faces in the order of their minus cells, so a run covers a compact set of cells).
// TMEM per warpgroup: D- [0, NE), D+ [NE, 2 NE) (coefficients overwrite them in place),
// Y- [2 NE, 2 NE + NI), Y+ [2 NE + NI, 2 NE + 2 NI).  The rows U-, U+ (the A operands of the
// evaluation GEMMs) are stored by each thread into its own lane of the Y columns, which the
// integration GEMMs overwrite only after the evaluation GEMMs have completed.
// Each side's values enter in the relabelled cell's DoF order (a permuted read of the staged row)
// and its results leave in the cell's own order (a permuted write to a row of shared memory, then
// vector reductions).  The DoF values of tile t+1 and the face data of tile t+2 are copied
// (cp.async) while tile t is computed.
template <int ND, int NQF, bool BF16>
__global__ void __launch_bounds__(kT * FaceShape<ND, NQF, BF16>::GMAX, 1)
    k_dg_face_tc(const int32_t* __restrict__ tcell, const int32_t* __restrict__ tperm, const float* __restrict__ tgeo,
                 const int8_t* __restrict__ dperm, const uint8_t* __restrict__ img, const float* __restrict__ u,
                 float* __restrict__ y, int64_t ntiles, uint32_t tmem_cols, int32_t* __restrict__ status) {
  using S = FaceShape<ND, NQF, BF16>;
  constexpr int AW = BF16 ? S::KE / 2 : S::KE;  // TMEM columns of one row of U
  static_assert(AW <= S::NI && AW % 8 == 0, "rows of U must fit in the Y columns");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int G = blockDim.x / kT;
  const int g = threadIdx.x / kT;
  const int m = threadIdx.x % kT;
  const int warp = threadIdx.x >> 5;
  uint8_t* misc = smem;
  uint8_t* sE = smem + 128;
  uint8_t* sI = sE + S::E_BYTES;
  int8_t* sP = reinterpret_cast<int8_t*>(sI + S::I_BYTES);  // [24][perm_row_bytes]
  uint8_t* wg = smem + face_cta_bytes<ND, NQF, BF16>() + size_t(g) * face_wg_bytes<ND, NQF, BF16>();
  float* sU = reinterpret_cast<float*>(wg);                         // [2 sides][128][ND] (own rows)
  float* sR = sU + 2 * kT * ND;                                      // [2 sides][128][ND] results
  uint32_t* sMeta = reinterpret_cast<uint32_t*>(sR + 2 * kT * ND);  // [2][kMetaWords]
  uint64_t* bar = reinterpret_cast<uint64_t*>(misc + 16 * g);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 64);
  const uint32_t bar_a = smem_u32(bar);
  {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(sE);
    for (int i = threadIdx.x; i < (S::E_BYTES + S::I_BYTES) / 16; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < 24 * perm_row_bytes<ND>(); i += blockDim.x) sP[i] = dperm[i];
  }
  if (m == 0) mbar_init(bar_a);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_proxy_async();  // the tables (generic writes) are read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + uint32_t(g * S::TCOLS);
  const uint32_t lane_base = tmem + (uint32_t((warp & 3) * 32) << 16);
  constexpr uint32_t YM = 2 * S::NE, YP = 2 * S::NE + S::NI;  // Y- / U- and Y+ / U+ columns
  const uint32_t aE = smem_u32(sE), aI = smem_u32(sI);
  const int64_t nw = int64_t(gridDim.x) * G;
  const int64_t per = (ntiles + nw - 1) / nw;
  const int64_t t0 = (int64_t(blockIdx.x) * G + g) * per;
  const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
  uint32_t phase = 0;
  bool failed = false;
  bool cells_done = false;
  if (t0 < t1) {
    // prologue: face data of t0, then the values of t0 and the face data of t0+1
    issue_face_meta(sMeta, tcell, tperm, tgeo, t0, m);
    cp_async_commit();
    cp_async_wait_group<0>();
    wg_sync(g);
    issue_face_u<ND>(sU, u, int64_t(int32_t(sMeta[m])), int64_t(int32_t(sMeta[kT + m])), m);
    if (t0 + 1 < t1) issue_face_meta(sMeta + kMetaWords, tcell, tperm, tgeo, t0 + 1, m);
    cp_async_commit();
  }
  for (int64_t t = t0; t < t1; ++t) {
    const int sl = int(t - t0) & 1;
    const uint32_t* meta = sMeta + sl * kMetaWords;
    uint32_t* meta_next = sMeta + (sl ^ 1) * kMetaWords;
    cp_async_wait_group<0>();  // this tile's values (own rows) and the next tile's face data
    wg_sync(g);
    // face data of the tile: cells of both sides, relabellings, a- a+ 2|F| tau
    const int64_t cm = int32_t(meta[m]), cp = int32_t(meta[kT + m]);
    const uint32_t rl = meta[2 * kT + m];
    const bool mirror = (rl & uint32_t(kMirrorFace)) != 0;  // boundary face: plus side = -(minus side)
    float geo[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) geo[r] = __uint_as_float(meta[(3 + r) * kT + m]);
    // 1. rows of U- and U+ in the relabelled DoF order (permuted reads of the staged rows, shifted
    //    by the minus side's first value) into this thread's TMEM lane
    uint32_t wm[perm_row_bytes<ND>() / 4], wp[perm_row_bytes<ND>() / 4];
    load_perm<ND>(sP, rl & 0xFFu, wm);
    load_perm<ND>(sP, (rl >> 8) & 0xFFu, wp);
    {
      float um[ND], up[ND];
      const float* rm = sU + m * ND;
      const float* rp = sU + (kT + m) * ND;
#pragma unroll
      for (int j = 0; j < ND; ++j) um[j] = rm[perm_at(wm, j)];
#pragma unroll
      for (int j = 0; j < ND; ++j) up[j] = mirror ? -um[j] : rp[perm_at(wp, j)];
      const float sh = um[0];
      uint32_t w[AW];
      pack_row<ND, S::KE, BF16>(um, sh, w);
      tmem_st_row<AW>(lane_base + YM, w);
      pack_row<ND, S::KE, BF16>(up, sh, w);
      tmem_st_row<AW>(lane_base + YP, w);
    }
    tmem_wait_st();
    tc_fence_before();
    wg_sync(g);
    // 2. evaluation GEMMs: value and reference gradient of both sides at the face's points
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int s2 = 0; s2 < S::KE / S::KSTEP; ++s2) {
        const uint64_t be = smem_desc(aE + s2 * 2 * S::LBO_E, S::LBO_E, 128);
        mma_ta<BF16>(tmem, tmem + YM + 8 * s2, be, S::idesc(S::NE), s2 > 0);
        mma_ta<BF16>(tmem + S::NE, tmem + YP + 8 * s2, be, S::idesc(S::NE), s2 > 0);
      }
      mma_commit(bar_a);
    }
    // prefetch: values of tile t+1 (this thread's rows of tile t are consumed) and face data of
    // tile t+2 (into the slot read above, before the barrier)
    if (t + 1 < t1) issue_face_u<ND>(sU, u, int64_t(int32_t(meta_next[m])), int64_t(int32_t(meta_next[kT + m])), m);
    if (t + 2 < t1) issue_face_meta(const_cast<uint32_t*>(meta), tcell, tperm, tgeo, t + 2, m);
    cp_async_commit();
    if (m == 0) failed |= !mbar_wait(bar_a, phase);
    phase ^= 1;
    failed = wg_any(g, failed);
    if (failed) break;
    tc_fence_after();
    // 3. SIPG flux per point (Eq. 2): coefficients of the test functions' values and reference
    //    gradients replace the evaluated values in TMEM, four points (16 columns) at a time
    {
      const float amx = geo[0], amy = geo[1], amz = geo[2], apx = geo[3], apy = geo[4], apz = geo[5];
      const float sF = geo[6], tau = geo[7];
#pragma unroll
      for (int c = 0; c < S::NE / 16; ++c) {
        uint32_t dm[16], dp[16];
        tmem_ld16(lane_base + 16 * c, dm);
        tmem_ld16(lane_base + S::NE + 16 * c, dp);
        tmem_wait_ld();
        reg_fence16(dm);
        reg_fence16(dp);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (4 * c + i < NQF) {
            const float vm = __uint_as_float(dm[4 * i]), vp = __uint_as_float(dp[4 * i]);
            const float dnm = fmaf(amx, __uint_as_float(dm[4 * i + 1]),
                                   fmaf(amy, __uint_as_float(dm[4 * i + 2]), amz * __uint_as_float(dm[4 * i + 3])));
            const float dnp = fmaf(apx, __uint_as_float(dp[4 * i + 1]),
                                   fmaf(apy, __uint_as_float(dp[4 * i + 2]), apz * __uint_as_float(dp[4 * i + 3])));
            const float jump = vm - vp;
            const float flux = sF * fmaf(0.5f, dnm + dnp, -tau * jump);  // 2|F| ({{dn u}} - tau [[u]])
            const float cd = -0.5f * sF * jump;
            dm[4 * i] = __float_as_uint(-flux);
            dm[4 * i + 1] = __float_as_uint(amx * cd);
            dm[4 * i + 2] = __float_as_uint(amy * cd);
            dm[4 * i + 3] = __float_as_uint(amz * cd);
            dp[4 * i] = __float_as_uint(flux);
            dp[4 * i + 1] = __float_as_uint(apx * cd);
            dp[4 * i + 2] = __float_as_uint(apy * cd);
            dp[4 * i + 3] = __float_as_uint(apz * cd);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) dm[4 * i + k] = dp[4 * i + k] = 0u;
          }
        }
        if constexpr (BF16) {
          uint32_t wm[8], wp[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            wm[i] = pack_bf16(__uint_as_float(dm[2 * i]), __uint_as_float(dm[2 * i + 1]));
            wp[i] = pack_bf16(__uint_as_float(dp[2 * i]), __uint_as_float(dp[2 * i + 1]));
          }
          tmem_st8(lane_base + 8 * c, wm);
          tmem_st8(lane_base + S::NE + 8 * c, wp);
        } else {
          tmem_st16(lane_base + 16 * c, dm);
          tmem_st16(lane_base + S::NE + 16 * c, dp);
        }
      }
    }
    tmem_wait_st();
    tc_fence_before();
    wg_sync(g);
    // 4. integration GEMMs (A = coefficients in TMEM, weights folded into the table); they
    //    overwrite the rows of U, whose GEMMs have completed
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int s2 = 0; s2 < S::KI / S::KSTEP; ++s2) {
        const uint64_t bi = smem_desc(aI + s2 * 2 * S::LBO_I, S::LBO_I, 128);
        mma_ta<BF16>(tmem + YM, tmem + 8 * s2, bi, S::idesc(S::NI), s2 > 0);
        mma_ta<BF16>(tmem + YP, tmem + S::NE + 8 * s2, bi, S::idesc(S::NI), s2 > 0);
      }
      mma_commit(bar_a);
      failed |= !mbar_wait(bar_a, phase);
    }
    phase ^= 1;
    failed = wg_any(g, failed);
    if (failed) break;
    tc_fence_after();
    // 5. both rows back in the cells' own DoF order and added to y (padding faces have 2|F| = 0),
    //    once the cell kernel before this one has written y
    if (!cells_done) {
      asm volatile("griddepcontrol.wait;" ::: "memory");
      cells_done = true;
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      uint32_t r[S::NI];
#pragma unroll
      for (int c = 0; c < S::NI / 16; ++c) tmem_ld16(lane_base + (side ? YP : YM) + 16 * c, r + 16 * c);
      tmem_wait_ld();
#pragma unroll
      for (int c = 0; c < S::NI / 16; ++c) reg_fence16(r + 16 * c);
      const uint32_t* pw = side ? wp : wm;
      float* row = sR + (side * kT + m) * ND;
#pragma unroll
      for (int j = 0; j < ND; ++j) row[perm_at(pw, j)] = __uint_as_float(r[j]);
      float vf[ND];
      load_row<ND>(row, vf);
      uint32_t v[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) v[j] = __float_as_uint(vf[j]);
      if (geo[6] != 0.0f && !(side && mirror)) red_cell<ND>(y + (side ? cp : cm) * ND, v);
    }
    tc_fence_before();
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(tmem_cols));
  if (failed && m == 0) atomicOr(status, 1);
}

template <int ND, int NQ, int NQF, bool BF16>
int launch_dg_tc(Ctx& c, const float* u, float* y, cudaStream_t st) {
  int dev = 0, smem_max = 0;
  TETMF_CK(cudaGetDevice(&dev));
  TETMF_CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  {
    // cell loop: as many warpgroups per CTA as TMEM and shared memory allow
    int G = cell_gmax<ND, NQ, BF16>();
    while (G > 1 && cell_smem<ND, NQ, BF16>(G) > size_t(smem_max)) --G;
    const size_t sm = cell_smem<ND, NQ, BF16>(G);
    if (sm > size_t(smem_max)) {
      set_error("DG tensor-core cell kernel does not fit on an SM (%zu bytes of shared memory)", sm);
      return FEM_EUNSUPPORTED;
    }
    auto kern = k_dg_cell_tc<ND, NQ, BF16>;
    if (int e = allow_smem(kern, sm)) return e;
    const uint32_t cols = uint32_t(pow2_cols(G * cell_tcols<ND, NQ, BF16>()));
    int64_t grid = (c.ntiles + G - 1) / G;
    if (grid > sm_count()) grid = sm_count();
    if (grid > 0) {
      kern<<<unsigned(grid), G * kT, sm, st>>>(c.d_metric32, static_cast<const uint8_t*>(BF16 ? c.d_tc_bf16 : c.d_tc_tf32),
                                               u, y, c.nc, c.ntiles, cols, c.d_status);
      TETMF_LAUNCH_CK();
    }
  }
  if (c.dg_ntiles > 0) {
    using S = FaceShape<ND, NQF, BF16>;
    int G = S::GMAX;
    while (G > 1 && face_cta_bytes<ND, NQF, BF16>() + G * face_wg_bytes<ND, NQF, BF16>() > size_t(smem_max)) --G;
    const size_t sm = face_cta_bytes<ND, NQF, BF16>() + G * face_wg_bytes<ND, NQF, BF16>();
    if (sm > size_t(smem_max)) {
      set_error("DG tensor-core face kernel does not fit on an SM (%zu bytes of shared memory)", sm);
      return FEM_EUNSUPPORTED;
    }
    auto kern = k_dg_face_tc<ND, NQF, BF16>;
    if (int e = allow_smem(kern, sm)) return e;
    const uint32_t cols = uint32_t(pow2_cols(G * S::TCOLS));
    int64_t grid = (c.dg_ntiles + G - 1) / G;
    if (grid > sm_count()) grid = sm_count();
    // may start while the cell kernel runs (it waits for it before adding to y)
    TETMF_CK(launch_early(kern, dim3(unsigned(grid)), dim3(unsigned(G * kT)), sm, st, c.d_dgt_cell, c.d_dgt_perm,
                          c.d_dgt_geo, c.d_dg_dperm,
                          static_cast<const uint8_t*>(BF16 ? c.d_dg_img_bf16 : c.d_dg_img_tf32), u, y, c.dg_ntiles,
                          cols, c.d_status));
    TETMF_LAUNCH_CK();
  }
  return FEM_OK;
}

}  // namespace

int dg_tc_prepare(Ctx& c) {
  // Every interior face is seen from both sides as local face 0 of a relabelled cell: new local
  // vertex 0 is the one opposite the face, new vertices 1, 2, 3 are the face's vertices in
  // increasing global order.  Both relabelled cells then place the face's quadrature points in the
  // same order, one evaluation and one integration table serve every face, and tiles may hold any
  // faces: they follow the minus cells' (Morton) order.  A relabelling is one of the 24
  // permutations s of the four local vertices (new vertex i = old vertex s[i], lexicographic
  // order of s); a new local DoF with multi-index b is the old one with multi-index b', b'[s[i]] = b[i].
  static const int kFv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  std::vector<std::array<int, 4>> perms;
  {
    std::array<int, 4> a = {0, 1, 2, 3};
    do perms.push_back(a);
    while (std::next_permutation(a.begin(), a.end()));
  }
  auto perm_id = [&](const std::array<int, 4>& s4) {
    return int(std::lower_bound(perms.begin(), perms.end(), s4) - perms.begin());
  };
  std::vector<std::array<int, 4>> nodes;  // local DoF order: multi-indices, lexicographic
  for (int b0 = 0; b0 <= c.p; ++b0)
    for (int b1 = 0; b1 <= c.p - b0; ++b1)
      for (int b2 = 0; b2 <= c.p - b0 - b1; ++b2) nodes.push_back({b0, b1, b2, c.p - b0 - b1 - b2});
  const int nd = c.nd;
  const int prow = (nd + 15) / 16 * 16;  // bytes per permutation row (16-byte aligned rows)
  std::vector<int8_t> dperm(size_t(24) * prow, 0);
  for (int id = 0; id < 24; ++id)
    for (int j = 0; j < nd; ++j) {
      std::array<int, 4> bo{};
      for (int i = 0; i < 4; ++i) bo[perms[id][i]] = nodes[j][i];
      dperm[size_t(id) * prow + j] = int8_t(std::find(nodes.begin(), nodes.end(), bo) - nodes.begin());
    }
  auto lib_cell = [&](int64_t e) { return &c.ucells[size_t(4) * c.cell_perm[e]]; };
  auto X = [&](int32_t v, int k) { return c.xyz[size_t(3) * v + k]; };
  // J'^-1 n for the cell relabelled by s (J' = [x_s1 - x_s0 | x_s2 - x_s0 | x_s3 - x_s0])
  auto jinv_n = [&](const int32_t* cv, const std::array<int, 4>& s4, const double n[3], double* a) {
    double J[3][3];
    for (int k = 0; k < 3; ++k)
      for (int col = 0; col < 3; ++col) J[k][col] = X(cv[s4[col + 1]], k) - X(cv[s4[0]], k);
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    // a = J^-1 n by Cramer's rule
    for (int col = 0; col < 3; ++col) {
      double M[3][3];
      for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) M[r][q] = q == col ? n[r] : J[r][q];
      a[col] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) /
               det;
    }
  };
  // interior faces (index i < nfi) and boundary faces (nfi + b) in the order of their minus cell
  // (then its local face).  A boundary face takes the mirror state of the weak Dirichlet condition,
  // u+ = -u-, d u+ / dn = d u- / dn: its plus side is the minus cell itself with negated values
  // (flag bit 16 of the relabelling word) and a+ = -a-, so that the interior flux gives the
  // boundary one, and only its minus side is added to y.
  const int64_t nf = c.nfi + c.nfb;
  auto minus_cell = [&](int64_t i) { return i < c.nfi ? c.fi_cell[i] : c.fb_cell[i - c.nfi]; };
  auto minus_face = [&](int64_t i) { return i < c.nfi ? (c.fi_code[i] & 3) : (c.fb_code[i - c.nfi] & 3); };
  std::vector<int64_t> order(nf);
  for (int64_t i = 0; i < nf; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const int32_t ca = minus_cell(a), cb = minus_cell(b);
    return ca < cb || (ca == cb && minus_face(a) < minus_face(b));
  });
  const int64_t nt = (nf + kT - 1) / kT;
  c.dg_ntiles = nt;
  std::vector<int32_t> cell(size_t(nt) * 2 * kT, 0), rl(size_t(nt) * kT, 0);
  std::vector<float> geo(size_t(nt) * 8 * kT, 0.0f);
  for (int64_t r = 0; r < nf; ++r) {
    const int64_t i = order[r], t = r / kT, m = r % kT;
    const bool mirror = i >= c.nfi;
    const int64_t ib = i - c.nfi;
    const int32_t em = minus_cell(i), ep = mirror ? em : c.fi_cell[c.nfi + i];
    const int fm = minus_face(i), fp = mirror ? fm : (c.fi_code[i] >> 2) & 3;
    const int32_t* vm = lib_cell(em);
    const int32_t* vp = lib_cell(ep);
    int32_t gv[3] = {vm[kFv[fm][0]], vm[kFv[fm][1]], vm[kFv[fm][2]]};
    std::sort(gv, gv + 3);
    std::array<int, 4> sm = {fm, 0, 0, 0}, sp = {fp, 0, 0, 0};
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 4; ++a) {
        if (vm[a] == gv[q]) sm[q + 1] = a;
        if (vp[a] == gv[q]) sp[q + 1] = a;
      }
    // unit normal out of the minus cell
    double e1[3], e2[3], n[3], o[3];
    for (int k = 0; k < 3; ++k) {
      e1[k] = X(gv[1], k) - X(gv[0], k);
      e2[k] = X(gv[2], k) - X(gv[0], k);
      o[k] = X(vm[fm], k) - X(gv[0], k);
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const double sgn = (n[0] * o[0] + n[1] * o[1] + n[2] * o[2]) > 0 ? -1.0 : 1.0;
    for (int k = 0; k < 3; ++k) n[k] *= sgn / len;
    double am[3], ap[3];
    jinv_n(vm, sm, n, am);
    if (mirror) {
      for (int k = 0; k < 3; ++k) ap[k] = -am[k];
    } else {
      jinv_n(vp, sp, n, ap);
    }
    cell[(size_t(t) * 2 + 0) * kT + m] = em;
    cell[(size_t(t) * 2 + 1) * kT + m] = ep;
    rl[size_t(t) * kT + m] = perm_id(sm) | (perm_id(sp) << 8) | (mirror ? kMirrorFace : 0);
    const double sF = mirror ? c.fb_geo[size_t(3) * c.nfb + ib] : c.fi_geo[size_t(6) * c.nfi + i];
    const double tau = mirror ? c.fb_geo[size_t(4) * c.nfb + ib] : c.fi_geo[size_t(7) * c.nfi + i];
    const double g8[8] = {am[0], am[1], am[2], ap[0], ap[1], ap[2], sF, tau};
    for (int q = 0; q < 8; ++q) geo[(size_t(t) * 8 + q) * kT + m] = float(g8[q]);
  }
  auto up = [&](auto** dst, const auto& v) -> int {
    using T = typename std::remove_reference<decltype(v[0])>::type;
    void* p = nullptr;
    TETMF_CK(cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(T)));
    c.allocations.push_back(p);
    if (!v.empty()) TETMF_CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = static_cast<std::remove_const_t<T>*>(p);
    return FEM_OK;
  };
  if (int s = up(&c.d_dgt_cell, cell)) return s;
  if (int s = up(&c.d_dgt_perm, rl)) return s;
  if (int s = up(&c.d_dgt_geo, geo)) return s;
  if (int s = up(&c.d_dg_dperm, dperm)) return s;
  switch (c.p) {
    case 1: return prepare_images<4, 4>(c);
    case 2: return prepare_images<10, 10>(c);
    case 3: return prepare_images<20, 20>(c);
    case 4: return prepare_images<35, 35>(c);
  }
  return FEM_OK;
}

}  // namespace tetmf

namespace tetmf {

int dg_apply_tc(Ctx& c, int prec, const void* u, void* y, void* stream) {
  if ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(y)) & 15u) {
    set_error("DG TF32/BF16 apply: u and y must be 16-byte aligned");
    return FEM_EINVAL;
  }
  cudaStream_t st = as_stream(stream);
  const float* uf = static_cast<const float*>(u);
  float* yf = static_cast<float*>(y);
  const bool bf = prec == FEM_BF16;
  if (bf) TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_dg_tc<ND, NQ, NQF, true>(c, uf, yf, st)))
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_dg_tc<ND, NQ, NQF, false>(c, uf, yf, st)))
}

}  // namespace tetmf
