// Inline-PTX helpers shared by the tcgen05 kernels (sm_103a): shared-memory
// operand descriptors, tcgen05.mma / commit / ld / st, mbarrier waits bounded
// by %globaltimer, cp.async, warpgroup barriers, and the host-side rounding of
// reference tables into TF32 / BF16 operand images.
//
// Shared-memory operand layout used throughout (K-major, no swizzle): a core
// matrix is 8 rows x 16 bytes stored contiguously; row r, column k of an
// operand with R rows sits at (k / KC) * LBO + (r / 8) * 128 + (r % 8) * 16 +
// (k % KC) * ES with KC = 16 / ES, SBO = 128 and LBO = (R / 8) * 128.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <vector>

namespace tetmf {
namespace {

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int pow2_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }
__host__ __device__ constexpr int max_i(int a, int b) { return a > b ? a : b; }

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
// the same, asking to be suspended until the phase completes or hint_ns have passed (a waiting warp
// then takes no issue slots from the warps that work)
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
constexpr uint32_t kSuspendHintNs = 200000;
// bounded wait: gives up after limit_ns (about 1 s) so that a lost completion cannot hang the GPU
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// the same with an abort flag shared by the CTA's waiters: the first wait that gives up raises it,
// and every other wait then returns at once (false)
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, volatile int* abort,
                                             uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait_hint(bar, parity, kSuspendHintNs)) {
    if (*abort) return false;
    if (global_ns() - t0 > limit_ns) {
      *abort = 1;
      return false;
    }
  }
  return true;
}
// a counter in shared memory that only grows, written with release and read with acquire semantics
// (CTA scope): unlike an mbarrier's phase parity it cannot alias when the writer runs ahead
__device__ __forceinline__ void st_release_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
// bounded wait until the counter reaches target (same limit and abort flag as mbar_wait_ab)
__device__ __forceinline__ bool count_wait_ab(uint32_t addr, uint32_t target, volatile int* abort,
                                              uint64_t limit_ns = kWaitLimitNs) {
  if (ld_acquire_u32(addr) >= target) return true;
  const uint64_t t0 = global_ns();
  while (ld_acquire_u32(addr) < target) {
    if (*abort) return false;
    if (global_ns() - t0 > limit_ns) {
      *abort = 1;
      return false;
    }
    __nanosleep(64);
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// TF32 high part of an FP32 value (the 19 bits the tensor core reads); value - high part is
// exact in FP32 and is the low part of a 3xTF32 split
__device__ __forceinline__ uint32_t tf32_hi(uint32_t bits) { return bits & 0xFFFFE000u; }

// write one K-major row (row m) of K values into a 128-row operand (LBO = 16 * 128)
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
      // FP32 bits as the TF32 operand (the tensor core reads the top 19 bits)
      w.x = __float_as_uint(v[c * 4 + 0]);
      w.y = __float_as_uint(v[c * 4 + 1]);
      w.z = __float_as_uint(v[c * 4 + 2]);
      w.w = __float_as_uint(v[c * 4 + 3]);
    }
    *reinterpret_cast<uint4*>(p + c * ((kTile / 8) * 128)) = w;
  }
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
template <bool BF16>
__device__ __forceinline__ void mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// barrier of the 128 threads of one warpgroup (named barrier 1 + g)
__device__ __forceinline__ void wg_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }
__device__ __forceinline__ bool wg_any(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, 128, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"(uint32_t(v)), "r"(1 + g)
      : "memory");
  return r != 0;
}

// Column order of the gradients G (GEMM 1 output) and of Q (GEMM 2 K index): quadrature points
// in pairs (q, q') = (2 p, 2 p + 1), six columns per pair, (x_q, x_q', y_q, y_q', z_q, z_q'), so
// that one packed FP32x2 instruction applies the metric to two points; an odd count leaves the
// last pair's second point as zero padding (zero table rows).
__host__ __device__ constexpr int grad_col(int q, int k) { return 6 * (q / 2) + 2 * k + (q % 2); }

// (x, x', y, y', z, z') <- M (x, y, z) for two points at once: t_x = m0 x + m1 y + m2 z,
// t_y = m1 x + m3 y + m4 z, t_z = m2 x + m4 y + m5 z (same rounding as the scalar fmaf chain);
// M0..M5 hold each metric entry in both halves
__device__ __forceinline__ void metric_pair(uint32_t* d, uint64_t M0, uint64_t M1, uint64_t M2, uint64_t M3,
                                            uint64_t M4, uint64_t M5) {
  asm("{\n\t.reg .b64 gx, gy, gz, tx, ty, tz;\n\t"
      "mov.b64 gx, {%0, %1};\n\tmov.b64 gy, {%2, %3};\n\tmov.b64 gz, {%4, %5};\n\t"
      "mul.rn.f32x2 tx, %8, gz;\n\tfma.rn.f32x2 tx, %7, gy, tx;\n\tfma.rn.f32x2 tx, %6, gx, tx;\n\t"
      "mul.rn.f32x2 ty, %10, gz;\n\tfma.rn.f32x2 ty, %9, gy, ty;\n\tfma.rn.f32x2 ty, %7, gx, ty;\n\t"
      "mul.rn.f32x2 tz, %11, gz;\n\tfma.rn.f32x2 tz, %10, gy, tz;\n\tfma.rn.f32x2 tz, %8, gx, tz;\n\t"
      "mov.b64 {%0, %1}, tx;\n\tmov.b64 {%2, %3}, ty;\n\tmov.b64 {%4, %5}, tz;\n\t}"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5])
      : "l"(M0), "l"(M1), "l"(M2), "l"(M3), "l"(M4), "l"(M5));
}
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(__float_as_uint(lo)), "r"(__float_as_uint(hi)));
  return r;
}
__device__ __forceinline__ uint64_t splat2(float v) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "r"(__float_as_uint(v)));
  return r;
}

// D_e of Eq. 3 for one cell (row m = the thread's TMEM lane): the reference gradients G in
// TMEM (columns in grad_col order) are replaced in place by Q = (k_q) M_e g_q, in chunks of 16
// points (8 pairs, 48 columns); columns past the last pair in the last chunk are zeroed.
// TF32: FP32 bits, one column per element; BF16: pairs packed into one column (Q column e / 2),
// which never overtakes the columns still to be read.  kq = this cell's coefficients at the NQ
// points, or null.  X3 (3xTF32): Q is split into a TF32 high part (kept in place) and the
// remainder (exact in FP32, stored at column offset qlo), for the three-product GEMM 2.
// CURVED: the metric differs per point; qm points at this cell's entry (q, r) = qm[(6 q + r) * 128]
// and a chunk's 96 values are loaded before its gradients are read from TMEM.
// ROLLED: the chunks are not unrolled (one chunk's 48 values live at a time; for kernels run at
// 128 registers per thread).
template <int ND, int NQ, bool BF16, bool HAS_K, bool X3 = false, bool CURVED = false, bool ROLLED = false>
__device__ __forceinline__ void metric_to_q(uint32_t lane_base, float m0, float m1, float m2, float m3, float m4,
                                            float m5, const float* kq, uint32_t qlo = 0,
                                            const float* __restrict__ qm = nullptr) {
  constexpr int NP = (NQ + 1) / 2;  // point pairs
  constexpr int NCHUNK = (NP + 7) / 8;
  const uint64_t M0 = splat2(m0), M1 = splat2(m1), M2 = splat2(m2), M3 = splat2(m3), M4 = splat2(m4),
                 M5 = splat2(m5);
  auto chunk = [&](int c) {
    const int np = (NP - 8 * c) < 8 ? (NP - 8 * c) : 8;  // pairs in this chunk
    const int nl = (6 * np + 15) / 16;                    // x16 loads in this chunk
    float mq[CURVED ? 96 : 1];
    if constexpr (CURVED) {
#pragma unroll
      for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int r = 0; r < 6; ++r)
          mq[6 * i + r] = 16 * c + i < NQ ? __ldcs(qm + (size_t(16 * c + i) * 6 + r) * kTile) : 0.0f;
    }
    uint32_t d[48];
#pragma unroll
    for (int l = 0; l < 3; ++l)
      if (l < nl) tmem_ld16(lane_base + 48 * c + 16 * l, d + 16 * l);
    tmem_wait_ld();
#pragma unroll
    for (int l = 0; l < 3; ++l)
      if (l < nl) reg_fence16(d + 16 * l);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < np) {
        if constexpr (CURVED) {
          const float* a = mq + 12 * i;  // point 2i of the chunk, then point 2i + 1
          metric_pair(d + 6 * i, pack2(a[0], a[6]), pack2(a[1], a[7]), pack2(a[2], a[8]), pack2(a[3], a[9]),
                      pack2(a[4], a[10]), pack2(a[5], a[11]));
        } else {
          metric_pair(d + 6 * i, M0, M1, M2, M3, M4, M5);
        }
        if constexpr (HAS_K) {
          const int q = 16 * c + 2 * i;
          const float k0 = kq[q], k1 = q + 1 < NQ ? kq[q + 1] : 0.0f;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            d[6 * i + 2 * a] = __float_as_uint(__uint_as_float(d[6 * i + 2 * a]) * k0);
            d[6 * i + 2 * a + 1] = __float_as_uint(__uint_as_float(d[6 * i + 2 * a + 1]) * k1);
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < 6; ++a)
          if (6 * i + a < 16 * nl) d[6 * i + a] = 0u;
      }
    }
    if constexpr (BF16) {
      uint32_t w[24];
#pragma unroll
      for (int i = 0; i < 24; ++i) w[i] = pack_bf16(__uint_as_float(d[2 * i]), __uint_as_float(d[2 * i + 1]));
#pragma unroll
      for (int l = 0; l < 3; ++l)
        if (l < nl) tmem_st8(lane_base + 24 * c + 8 * l, w + 8 * l);
    } else {
#pragma unroll
      for (int l = 0; l < 3; ++l)
        if (l < nl) {
          if constexpr (X3) {
            uint32_t lo[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const uint32_t h = tf32_hi(d[16 * l + i]);
              lo[i] = __float_as_uint(__uint_as_float(d[16 * l + i]) - __uint_as_float(h));
              d[16 * l + i] = h;
            }
            tmem_st16(lane_base + qlo + 48 * c + 16 * l, lo);
          }
          tmem_st16(lane_base + 48 * c + 16 * l, d + 16 * l);
        }
    }
  };
  if constexpr (ROLLED) {
#pragma unroll 1
    for (int c = 0; c < NCHUNK; ++c) chunk(c);
  } else {
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c) chunk(c);
  }
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

// shapes of the two cell GEMMs (difference form) and of their TMEM columns; see cg_tc.cu
template <int ND, int NQ, bool BF16>
struct TcShape {
  static constexpr int ES = BF16 ? 2 : 4;
  static constexpr int KC = 16 / ES;
  static constexpr int KSTEP = 2 * KC;
  static constexpr int N3 = 6 * ((NQ + 1) / 2);  // gradient columns in grad_col order (pairs of points)
  static constexpr int ND1 = ND - 1;  // DoFs 1..nd-1 enter as differences to DoF 0
  static constexpr int K1 = round_up(ND1, KSTEP);
  static constexpr int N1 = round_up(N3, 16);
  static constexpr int K2 = round_up(N3, KSTEP);
  static constexpr int N2 = round_up(ND1, 16);
  // TMEM: G in columns [0, N1); Q overwrites it in place (TF32: one column per
  // element; BF16: packed pairs, QW = N1 / 2 columns); Y' in [N1, N1 + N2)
  static constexpr int QW = BF16 ? N1 / 2 : N1;
  static constexpr int D2_COL = N1;  // Y' is read while GEMM 1 of the next tile writes G
  static constexpr int COLS = pow2_cols(N1 + N2);
  static constexpr int LBO_A = (kTile / 8) * 128;
  static constexpr int LBO_B1 = (N1 / 8) * 128;
  static constexpr int LBO_B2 = (N2 / 8) * 128;
  static constexpr int A1_BYTES = kTile * K1 * ES;
  static constexpr int A2_BYTES = kTile * K2 * ES;
  static constexpr int B1_BYTES = N1 * K1 * ES;
  static constexpr int B2_BYTES = N2 * K2 * ES;
  // instruction descriptor (kind::tf32 / kind::f16): D = F32 (bits 4-5 = 1),
  // A/B format (bits 7-9, 10-12) = TF32 (2) or BF16 (1), both K-major,
  // N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t fmt = BF16 ? 1u : 2u;
  __host__ __device__ static constexpr uint32_t idesc(int n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kTile >> 4) << 24);
  }
  static_assert(N1 % 16 == 0 && N1 >= 16 && N1 <= 256, "GEMM 1 N out of range");
  static_assert(N2 % 16 == 0 && N2 >= 16 && N2 <= 256, "GEMM 2 N out of range");
};

}  // namespace
}  // namespace tetmf
