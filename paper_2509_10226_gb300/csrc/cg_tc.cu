// Continuous-Galerkin apply with the interpolation products on the 5th-generation
// tensor cores (tcgen05, sm_103a), TF32 or BF16 operands with FP32 accumulation.
//
// The two dense contractions of Eq. 3 for a batch of 128 cells become GEMMs
// ("matrix-matrix product", Sec. 2.4, with the batch extended from 4 x n_lanes
// cells to 128 cells = the M of one tcgen05.mma):
//   GEMM 1:  G[128 x 3nq]  = U'[128 x nd-1] . E'^T   (E' = columns 1..nd-1 of E, Eq. 4;
//                                                     U'[m, j-1] = u_j - u_0 of cell m)
//   D_e:     Q[m, 3q+k]    = w_q k_q (M_e G[m, 3q:3q+3])_k    per thread (row m)
//   GEMM 2:  Y'[128 x nd-1] = Q[128 x 3nq] . E',      y_0 = -sum_{j>=1} y_j
// The difference form is E u_e rewritten with sum_j E_j = 0 (partition of
// unity); it is exact for exact tables and keeps rounded TF32/BF16 tables
// consistent (constants map to zero, operand error relative to the gradient).
// A CTA of 128 threads owns one TMEM lane per cell.  Per tile:
//   1. each thread gathers its cell's DoFs (masked gather) and writes its row
//      of U into shared memory in the canonical K-major no-swizzle layout;
//   2. one thread issues GEMM 1 (tcgen05.mma, D in TMEM) and commits to an
//      mbarrier;
//   3. each thread reads its row of G from TMEM (tcgen05.ld 32x32b), applies
//      the 3x3 metric per quadrature point in FP32 and writes its row of Q;
//   4. one thread issues GEMM 2 into the same TMEM columns;
//   5. each thread reads its row of Y and scatter-adds it (atomics, G_e^T).
// E^T and E are staged once per persistent CTA from pre-laid-out byte images.
//
// Shared-memory operand layout (K-major, no swizzle): a core matrix is 8 rows
// x 16 bytes, stored contiguously; row r, column k of an operand with R rows
// sits at  (k / KC) * LBO + (r / 8) * 128 + (r % 8) * 16 + (k % KC) * ES,
// KC = 16 / ES elements per core-matrix row, SBO = 128 (next 8 rows),
// LBO = (R / 8) * 128 (next 16-byte column block).  One MMA consumes K = 2 KC.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kT = kTile;

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int pow2_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }
__host__ __device__ constexpr int max_i(int a, int b) { return a > b ? a : b; }

template <int ND, int NQ, bool BF16>
struct TcShape {
  static constexpr int ES = BF16 ? 2 : 4;
  static constexpr int KC = 16 / ES;
  static constexpr int KSTEP = 2 * KC;
  static constexpr int N3 = 3 * NQ;
  static constexpr int ND1 = ND - 1;  // DoFs 1..nd-1 enter as differences to DoF 0
  static constexpr int K1 = round_up(ND1, KSTEP);
  static constexpr int N1 = round_up(N3, 16);
  static constexpr int K2 = round_up(N3, KSTEP);
  static constexpr int N2 = round_up(ND1, 16);
  static constexpr int COLS = pow2_cols(max_i(N1, N2));
  static constexpr int LBO_A = (kT / 8) * 128;
  static constexpr int LBO_B1 = (N1 / 8) * 128;
  static constexpr int LBO_B2 = (N2 / 8) * 128;
  static constexpr int A1_BYTES = kT * K1 * ES;
  static constexpr int A2_BYTES = kT * K2 * ES;
  static constexpr int B1_BYTES = N1 * K1 * ES;
  static constexpr int B2_BYTES = N2 * K2 * ES;
  // instruction descriptor (kind::tf32 / kind::f16): D = F32 (bits 4-5 = 1),
  // A/B format (bits 7-9, 10-12) = TF32 (2) or BF16 (1), both K-major,
  // N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t fmt = BF16 ? 1u : 2u;
  __host__ __device__ static constexpr uint32_t idesc(int n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kT >> 4) << 24);
  }
  static_assert(N1 % 16 == 0 && N1 >= 16 && N1 <= 256, "GEMM 1 N out of range");
  static_assert(N2 % 16 == 0 && N2 >= 16 && N2 <= 256, "GEMM 2 N out of range");
};

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: gives up after ~1 s so that a lost completion cannot hang the GPU
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > 1000000000ull) return false;
  return true;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45), version 1 (46-47),
  // base offset 0, layout SWIZZLE_NONE (61-63 = 0)
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}
template <bool BF16>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// keeps every use of the loaded registers after tcgen05.wait::ld
__device__ __forceinline__ void reg_fence16(uint32_t* r) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
}
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// write one K-major row (row m) of K values into an operand with LBO = LBO_A
template <int K, bool BF16>
__device__ __forceinline__ void write_row(uint8_t* base, int m, const float* v) {
  constexpr int KC = BF16 ? 8 : 4;
  uint8_t* p = base + (m / 8) * 128 + (m % 8) * 16;
#pragma unroll
  for (int c = 0; c < K / KC; ++c) {
    uint4 w;
    if constexpr (BF16) {
      w.x = pack_bf16(v[c * 8 + 0], v[c * 8 + 1]);
      w.y = pack_bf16(v[c * 8 + 2], v[c * 8 + 3]);
      w.z = pack_bf16(v[c * 8 + 4], v[c * 8 + 5]);
      w.w = pack_bf16(v[c * 8 + 6], v[c * 8 + 7]);
    } else {
      w.x = to_tf32(v[c * 4 + 0]);
      w.y = to_tf32(v[c * 4 + 1]);
      w.z = to_tf32(v[c * 4 + 2]);
      w.w = to_tf32(v[c * 4 + 3]);
    }
    *reinterpret_cast<uint4*>(p + c * ((kT / 8) * 128)) = w;
  }
}

constexpr int kMaxNQ = 70;

template <int ND, int NQ, bool BF16>
__global__ void __launch_bounds__(kT, 1)
    k_cg_apply_tc(const int32_t* __restrict__ idx, const float* __restrict__ metric, const float* __restrict__ tabW,
                  const uint8_t* __restrict__ bimg, const float* __restrict__ u, float* __restrict__ y,
                  const float* __restrict__ kcoef, int64_t nc, int64_t ntiles, int32_t* __restrict__ status) {
  using S = TcShape<ND, NQ, BF16>;
  constexpr int KS = NQ | 1;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA2 = smem;
  uint8_t* sA1 = sA2 + S::A2_BYTES;
  uint8_t* sB1 = sA1 + S::A1_BYTES;
  uint8_t* sB2 = sB1 + S::B1_BYTES;
  float* sw = reinterpret_cast<float*>(sB2 + S::B2_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sw + round_up(NQ, 4));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  float* sk = reinterpret_cast<float*>(tslot + 4);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  {
    const uint4* src = reinterpret_cast<const uint4*>(bimg);
    uint4* dst = reinterpret_cast<uint4*>(sB1);
    for (int i = tid; i < (S::B1_BYTES + S::B2_BYTES) / 16; i += kT) dst[i] = src[i];
  }
  for (int i = tid; i < NQ; i += kT) sw[i] = tabW[i];
  const uint32_t bar_a = smem_u32(bar);
  if (tid == 0) mbar_init(bar_a);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(uint32_t(S::COLS)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = tmem + (uint32_t(warp * 32) << 16);
  const uint32_t aA1 = smem_u32(sA1), aA2 = smem_u32(sA2), aB1 = smem_u32(sB1), aB2 = smem_u32(sB2);
  uint32_t phase = 0;
  bool failed = false;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t cell0 = tile * kT;
    const int m = tid;
    const bool active = cell0 + m < nc;
    if (kcoef) {
      const int64_t ncell = nc - cell0 < kT ? nc - cell0 : kT;
      const float* src = kcoef + cell0 * NQ;
      for (int64_t i = tid; i < ncell * NQ; i += kT) sk[(i / NQ) * KS + i % NQ] = src[i];
    }
    // 1. masked gather of the cell's DoFs into row m of U
    int g[ND];
    float ue[ND], v1[S::K1];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      g[j] = active ? __ldg(idx + (tile * ND + j) * kT + m) : -1;
      ue[j] = g[j] >= 0 ? __ldg(u + g[j]) : 0.0f;
    }
    // sum_j E_j = 0 (the gradients of a partition of unity), so E u_e equals
    // E' (u_j - u_0)_{j >= 1} with E' the columns 1..nd-1 of E; rounding the
    // differences and E' keeps constants in the kernel exactly and makes the
    // operand error relative to the gradient instead of to u
#pragma unroll
    for (int j = 1; j < ND; ++j) v1[j - 1] = ue[j] - ue[0];
#pragma unroll
    for (int j = S::ND1; j < S::K1; ++j) v1[j] = 0.0f;
    write_row<S::K1, BF16>(sA1, m, v1);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // 2. GEMM 1
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < S::K1 / S::KSTEP; ++s)
        mma<BF16>(tmem, smem_desc(aA1 + s * 2 * S::LBO_A, S::LBO_A, 128),
                  smem_desc(aB1 + s * 2 * S::LBO_B1, S::LBO_B1, 128), S::idesc(S::N1), s > 0);
      mma_commit(bar_a);
    }
    failed |= !mbar_wait(bar_a, phase);
    phase ^= 1;
    if (__syncthreads_or(failed)) break;
    tc_fence_after();
    // 3. D_e at the quadrature points: row m of G from TMEM, metric, row m of Q
    uint32_t d[S::N1];
#pragma unroll
    for (int c = 0; c < S::N1 / 16; ++c) tmem_ld16(lane_base + c * 16, d + c * 16);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < S::N1 / 16; ++c) reg_fence16(d + c * 16);
    const float* mp = metric + tile * 6 * kT + m;
    const float m0 = mp[0], m1 = mp[kT], m2 = mp[2 * kT], m3 = mp[3 * kT], m4 = mp[4 * kT], m5 = mp[5 * kT];
    float v2[S::K2];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float gx = __uint_as_float(d[3 * q]), gy = __uint_as_float(d[3 * q + 1]),
                  gz = __uint_as_float(d[3 * q + 2]);
      float cq = sw[q];
      if (kcoef) cq *= sk[m * KS + q];
      v2[3 * q] = cq * fmaf(m0, gx, fmaf(m1, gy, m2 * gz));
      v2[3 * q + 1] = cq * fmaf(m1, gx, fmaf(m3, gy, m4 * gz));
      v2[3 * q + 2] = cq * fmaf(m2, gx, fmaf(m4, gy, m5 * gz));
    }
#pragma unroll
    for (int n = S::N3; n < S::K2; ++n) v2[n] = 0.0f;
    write_row<S::K2, BF16>(sA2, m, v2);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // 4. GEMM 2 into the same TMEM columns (all reads of G are complete)
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < S::K2 / S::KSTEP; ++s)
        mma<BF16>(tmem, smem_desc(aA2 + s * 2 * S::LBO_A, S::LBO_A, 128),
                  smem_desc(aB2 + s * 2 * S::LBO_B2, S::LBO_B2, 128), S::idesc(S::N2), s > 0);
      mma_commit(bar_a);
    }
    failed |= !mbar_wait(bar_a, phase);
    phase ^= 1;
    if (__syncthreads_or(failed)) break;
    tc_fence_after();
    // 5. row m of Y, scatter-add (G_e^T)
    uint32_t r[S::N2];
#pragma unroll
    for (int c = 0; c < S::N2 / 16; ++c) tmem_ld16(lane_base + c * 16, r + c * 16);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < S::N2 / 16; ++c) reg_fence16(r + c * 16);
    // y_0 = -sum_{j >= 1} y_j (same identity on the test side)
    float y0 = 0.0f;
#pragma unroll
    for (int j = 1; j < ND; ++j) {
      const float yj = __uint_as_float(r[j - 1]);
      y0 -= yj;
      if (g[j] >= 0) atomicAdd(y + g[j], yj);
    }
    if (g[0] >= 0) atomicAdd(y + g[0], y0);
    tc_fence_before();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(S::COLS)));
  if (failed && tid == 0) atomicOr(status, 1);
}

// host: byte image of an operand stored K-major without swizzle
template <bool BF16>
void put_elem(std::vector<uint8_t>& img, size_t off, double v) {
  float f = float(v);
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  if (BF16) {
    // round to nearest even
    const uint32_t lsb = (bits >> 16) & 1u;
    const uint16_t h = uint16_t((bits + 0x7FFFu + lsb) >> 16);
    std::memcpy(&img[off], &h, 2);
  } else {
    // TF32, round to nearest with ties away from zero (as cvt.rna.tf32.f32)
    bits = (bits + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&img[off], &bits, 4);
  }
}

template <int ND, int NQ, bool BF16>
std::vector<uint8_t> b_image(const RefTables& t) {
  using S = TcShape<ND, NQ, BF16>;
  std::vector<uint8_t> img(S::B1_BYTES + S::B2_BYTES, 0);
  auto off = [](int r, int k, int lbo) {
    return size_t((k / S::KC) * lbo + (r / 8) * 128 + (r % 8) * 16 + (k % S::KC) * S::ES);
  };
  // B1 = E' as [N1 rows = 3q+k][K1 = j-1]; B2 = E'^T as [N2 rows = j-1][K2 = 3q+k]
  for (int n = 0; n < S::N3; ++n)
    for (int j = 1; j < ND; ++j) {
      const double e = t.E[size_t(n) * ND + j];
      put_elem<BF16>(img, off(n, j - 1, S::LBO_B1), e);
      put_elem<BF16>(img, S::B1_BYTES + off(j - 1, n, S::LBO_B2), e);
    }
  return img;
}

template <int ND, int NQ, bool BF16>
size_t tc_smem(bool with_k) {
  using S = TcShape<ND, NQ, BF16>;
  size_t b = size_t(S::A2_BYTES) + S::A1_BYTES + S::B1_BYTES + S::B2_BYTES + round_up(NQ, 4) * 4 + 8 + 16;
  if (with_k) b += size_t(kT) * (NQ | 1) * 4;
  return b;
}

template <int ND, int NQ, bool BF16>
int upload_image(Ctx& c, void** dst) {
  const std::vector<uint8_t> img = b_image<ND, NQ, BF16>(c.tab);
  void* p = nullptr;
  TETMF_CK(cudaMalloc(&p, img.size()));
  c.allocations.push_back(p);
  TETMF_CK(cudaMemcpy(p, img.data(), img.size(), cudaMemcpyHostToDevice));
  *dst = p;
  return FEM_OK;
}

template <int ND, int NQ>
int prepare(Ctx& c) {
  if (int s = upload_image<ND, NQ, false>(c, &c.d_tc_tf32)) return s;
  return upload_image<ND, NQ, true>(c, &c.d_tc_bf16);
}

template <int ND, int NQ, bool BF16>
int launch(Ctx& c, const float* u, float* y, const float* k, cudaStream_t st) {
  if (int e = init_rows<float>(y, u, c.d_mask, c.ndofs, 0.0f, st)) return e;
  const size_t sm = tc_smem<ND, NQ, BF16>(k != nullptr);
  auto kern = k_cg_apply_tc<ND, NQ, BF16>;
  if (int e = allow_smem(kern, sm)) return e;
  TETMF_CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int per_sm = 0;
  TETMF_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, sm));
  if (per_sm < 1) {
    set_error("tensor-core kernel does not fit on an SM (%zu bytes of shared memory)", sm);
    return FEM_ECUDA;
  }
  const int cols = TcShape<ND, NQ, BF16>::COLS;
  if (per_sm * cols > 512) per_sm = 512 / cols;
  int64_t grid = int64_t(sm_count()) * per_sm;
  if (grid > c.ntiles) grid = c.ntiles;
  const TableLayout L = tables_layout(c.tab);
  const void* img = BF16 ? c.d_tc_bf16 : c.d_tc_tf32;
  kern<<<unsigned(grid), kT, sm, st>>>(c.d_idx, c.d_metric32, c.d_tab32 + L.w, static_cast<const uint8_t*>(img), u, y,
                                       k, c.nc, c.ntiles, c.d_status);
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

}  // namespace

int tc_prepare(Ctx& c) {
  switch (c.p) {
    case 1: return prepare<4, 5>(c);
    case 2: return prepare<10, 15>(c);
    case 3: return prepare<20, 35>(c);
    case 4: return prepare<35, 70>(c);
  }
  return FEM_OK;
}

int cg_apply_tc(Ctx& c, int prec, const void* u, void* y, const void* k, void* stream) {
  cudaStream_t st = as_stream(stream);
  const float* uf = static_cast<const float*>(u);
  float* yf = static_cast<float*>(y);
  const float* kf = static_cast<const float*>(k);
  const bool bf = prec == FEM_BF16;
  switch (c.p) {
    case 1: return bf ? launch<4, 5, true>(c, uf, yf, kf, st) : launch<4, 5, false>(c, uf, yf, kf, st);
    case 2: return bf ? launch<10, 15, true>(c, uf, yf, kf, st) : launch<10, 15, false>(c, uf, yf, kf, st);
    case 3: return bf ? launch<20, 35, true>(c, uf, yf, kf, st) : launch<20, 35, false>(c, uf, yf, kf, st);
    case 4: return bf ? launch<35, 70, true>(c, uf, yf, kf, st) : launch<35, 70, false>(c, uf, yf, kf, st);
  }
  set_error("degree %d not supported", c.p);
  return FEM_EUNSUPPORTED;
}

}  // namespace tetmf
