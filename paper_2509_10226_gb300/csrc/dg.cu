// Discontinuous Galerkin (SIPG) operator, Eq. 2 evaluated as Eq. 5: a cell loop
// (Eq. 3 on per-cell DoFs) followed by a loop over interior faces and one over
// boundary faces.
//
// DoFs of a cell are contiguous (u[c*nd + j]), so only one index per cell is
// needed (Sec. 2.3, Eq. 7).  The cell kernel stages the tile's 128 x nd block
// of u through shared memory (one fully coalesced load) and writes y the same
// way, without atomics.  Face kernels run one thread per face: values and
// reference gradients of both sides at the face quadrature points come from
// per-local-face tables (the + side reads them through the orientation
// permutation of the face points), the normal derivative is a.grad_hat with
// a = J^-1 n precomputed per face and side, and the flux
//   v-:  -(1/2) dn v [[u]] - v ({{dn u}} - tau [[u]])
//   v+:  -(1/2) dn v [[u]] + v ({{dn u}} - tau [[u]])
// is integrated back and added to both cells with atomics.  Boundary faces use
// the mirror state u+ = -u-, grad u+ = grad u- (homogeneous Dirichlet).
#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kT = kTile;

template <int ND, int NQ, typename T>
__global__ void __launch_bounds__(kT) k_dg_cell(const T* __restrict__ metric, const T* __restrict__ tabE,
                                                const T* __restrict__ tabW, const T* __restrict__ u,
                                                T* __restrict__ y, int64_t nc) {
  constexpr int RS = ND | 1;  // odd row stride of the staged tile
  extern __shared__ __align__(16) unsigned char smem[];
  T* sE = reinterpret_cast<T*>(smem);
  T* sw = sE + NQ * 3 * ND;
  T* su = sw + NQ;
  for (int i = threadIdx.x; i < NQ * 3 * ND; i += kT) sE[i] = tabE[i];
  for (int i = threadIdx.x; i < NQ; i += kT) sw[i] = tabW[i];
  const int64_t tile = blockIdx.x;
  const int64_t cell0 = tile * kT;
  const int ncell = int(nc - cell0 < kT ? nc - cell0 : kT);
  const T* src = u + cell0 * ND;
  for (int i = threadIdx.x; i < ncell * ND; i += kT) su[(i / ND) * RS + i % ND] = src[i];
  __syncthreads();
  const int lane = threadIdx.x;
  if (lane < ncell) {
    T ue[ND], ye[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      ue[j] = su[lane * RS + j];
      ye[j] = T(0);
    }
    const T* mp = metric + tile * 6 * kT + lane;
    const T m0 = mp[0], m1 = mp[kT], m2 = mp[2 * kT], m3 = mp[3 * kT], m4 = mp[4 * kT], m5 = mp[5 * kT];
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      const T* Eq = sE + q * 3 * ND;
      T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        gx = fma(Eq[j], ue[j], gx);
        gy = fma(Eq[ND + j], ue[j], gy);
        gz = fma(Eq[2 * ND + j], ue[j], gz);
      }
      const T c = sw[q];
      const T tx = c * fma(m0, gx, fma(m1, gy, m2 * gz));
      const T ty = c * fma(m1, gx, fma(m3, gy, m4 * gz));
      const T tz = c * fma(m2, gx, fma(m4, gy, m5 * gz));
#pragma unroll
      for (int j = 0; j < ND; ++j) ye[j] = fma(Eq[j], tx, fma(Eq[ND + j], ty, fma(Eq[2 * ND + j], tz, ye[j])));
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) su[lane * RS + j] = ye[j];
  }
  __syncthreads();
  T* dst = y + cell0 * ND;
  for (int i = threadIdx.x; i < ncell * ND; i += kT) dst[i] = su[(i / ND) * RS + i % ND];
}

template <int ND, int NQF, typename T>
struct FaceTables {
  T* V;    // [4][NQF][ND]
  T* G;    // [4][NQF][3][ND]
  T* w;    // [NQF]
  int* perm;  // [6][NQF]
};

template <int ND, int NQF, typename T>
__device__ inline FaceTables<ND, NQF, T> load_face_tables(unsigned char* raw, const T* __restrict__ Vf,
                                                          const T* __restrict__ Ef, const T* __restrict__ wf,
                                                          const int32_t* __restrict__ fperm) {
  FaceTables<ND, NQF, T> t;
  t.V = reinterpret_cast<T*>(raw);
  t.G = t.V + 4 * NQF * ND;
  t.w = t.G + 4 * NQF * 3 * ND;
  t.perm = reinterpret_cast<int*>(t.w + NQF);
  for (int i = threadIdx.x; i < 4 * NQF * ND; i += blockDim.x) t.V[i] = Vf[i];
  for (int i = threadIdx.x; i < 4 * NQF * 3 * ND; i += blockDim.x) t.G[i] = Ef[i];
  for (int i = threadIdx.x; i < NQF; i += blockDim.x) t.w[i] = wf[i];
  for (int i = threadIdx.x; i < 6 * NQF; i += blockDim.x) t.perm[i] = fperm[i];
  return t;
}

// value and normal derivative (a . grad_hat u) of one side at face point q
template <int ND, typename T>
__device__ inline void eval_side(const T* __restrict__ V, const T* __restrict__ G, const T (&ue)[ND], T ax, T ay,
                                 T az, T& val, T& dn) {
  T v = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    v = fma(V[j], ue[j], v);
    gx = fma(G[j], ue[j], gx);
    gy = fma(G[ND + j], ue[j], gy);
    gz = fma(G[2 * ND + j], ue[j], gz);
  }
  val = v;
  dn = fma(ax, gx, fma(ay, gy, az * gz));
}

// ye += cv * V + cd * (a . G)
template <int ND, typename T>
__device__ inline void integrate_side(const T* __restrict__ V, const T* __restrict__ G, T cv, T bx, T by, T bz,
                                      T (&ye)[ND]) {
#pragma unroll
  for (int j = 0; j < ND; ++j) ye[j] = fma(cv, V[j], fma(bx, G[j], fma(by, G[ND + j], fma(bz, G[2 * ND + j], ye[j]))));
}

template <int ND, int NQF, typename T>
__global__ void __launch_bounds__(kT) k_dg_face_interior(const int32_t* __restrict__ fcell,
                                                         const int32_t* __restrict__ fcode,
                                                         const T* __restrict__ fgeo, const T* __restrict__ Vf,
                                                         const T* __restrict__ Ef, const T* __restrict__ wf,
                                                         const int32_t* __restrict__ fperm, const T* __restrict__ u,
                                                         T* __restrict__ y, int64_t nf) {
  extern __shared__ __align__(16) unsigned char smem[];
  const FaceTables<ND, NQF, T> tb = load_face_tables<ND, NQF, T>(smem, Vf, Ef, wf, fperm);
  __syncthreads();
  const int64_t f = blockIdx.x * int64_t(kT) + threadIdx.x;
  if (f >= nf) return;
  const int64_t cm = fcell[f], cp = fcell[nf + f];
  const int code = fcode[f];
  const int fm = code & 3, fp = (code >> 2) & 3, o = code >> 4;
  const T amx = fgeo[f], amy = fgeo[nf + f], amz = fgeo[2 * nf + f];
  const T apx = fgeo[3 * nf + f], apy = fgeo[4 * nf + f], apz = fgeo[5 * nf + f];
  const T s = fgeo[6 * nf + f], tau = fgeo[7 * nf + f];
  T um[ND], up[ND], ym[ND], yp[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    um[j] = u[cm * ND + j];
    up[j] = u[cp * ND + j];
    ym[j] = T(0);
    yp[j] = T(0);
  }
#pragma unroll 1
  for (int q = 0; q < NQF; ++q) {
    const int qp = tb.perm[o * NQF + q];
    const T* Vm = tb.V + (fm * NQF + q) * ND;
    const T* Gm = tb.G + (fm * NQF + q) * 3 * ND;
    const T* Vp = tb.V + (fp * NQF + qp) * ND;
    const T* Gp = tb.G + (fp * NQF + qp) * 3 * ND;
    T vm, dnm, vp, dnp;
    eval_side<ND, T>(Vm, Gm, um, amx, amy, amz, vm, dnm);
    eval_side<ND, T>(Vp, Gp, up, apx, apy, apz, vp, dnp);
    const T W = tb.w[q] * s;
    const T jump = vm - vp;
    const T flux = W * fma(T(0.5), dnm + dnp, -tau * jump);  // W ({{dn u}} - tau [[u]])
    const T cd = T(-0.5) * W * jump;
    integrate_side<ND, T>(Vm, Gm, -flux, amx * cd, amy * cd, amz * cd, ym);
    integrate_side<ND, T>(Vp, Gp, flux, apx * cd, apy * cd, apz * cd, yp);
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    atomicAdd(y + cm * ND + j, ym[j]);
    atomicAdd(y + cp * ND + j, yp[j]);
  }
}

template <int ND, int NQF, typename T>
__global__ void __launch_bounds__(kT) k_dg_face_boundary(const int32_t* __restrict__ fcell,
                                                         const int32_t* __restrict__ fcode,
                                                         const T* __restrict__ fgeo, const T* __restrict__ Vf,
                                                         const T* __restrict__ Ef, const T* __restrict__ wf,
                                                         const int32_t* __restrict__ fperm, const T* __restrict__ u,
                                                         T* __restrict__ y, int64_t nf) {
  extern __shared__ __align__(16) unsigned char smem[];
  const FaceTables<ND, NQF, T> tb = load_face_tables<ND, NQF, T>(smem, Vf, Ef, wf, fperm);
  __syncthreads();
  const int64_t f = blockIdx.x * int64_t(kT) + threadIdx.x;
  if (f >= nf) return;
  const int64_t cm = fcell[f];
  const int fm = fcode[f] & 3;
  const T ax = fgeo[f], ay = fgeo[nf + f], az = fgeo[2 * nf + f];
  const T s = fgeo[3 * nf + f], tau = fgeo[4 * nf + f];
  T um[ND], ym[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    um[j] = u[cm * ND + j];
    ym[j] = T(0);
  }
#pragma unroll 1
  for (int q = 0; q < NQF; ++q) {
    const T* Vm = tb.V + (fm * NQF + q) * ND;
    const T* Gm = tb.G + (fm * NQF + q) * 3 * ND;
    T vm, dnm;
    eval_side<ND, T>(Vm, Gm, um, ax, ay, az, vm, dnm);
    const T W = tb.w[q] * s;
    // mirror state: [[u]] = 2 u-, {{dn u}} = dn u-
    const T jump = T(2) * vm;
    const T flux = W * fma(-tau, jump, dnm);
    const T cd = T(-0.5) * W * jump;
    integrate_side<ND, T>(Vm, Gm, -flux, ax * cd, ay * cd, az * cd, ym);
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) atomicAdd(y + cm * ND + j, ym[j]);
}

template <int ND, int NQ, int NQF, typename T>
int launch_dg(Ctx& c, const T* u, T* y, const T* metric, const T* tab, const T* fgi, const T* fgb, cudaStream_t st) {
  const TableLayout L = tables_layout(c.tab);
  const size_t sm_cell = (size_t(NQ) * 3 * ND + NQ + size_t(kT) * (ND | 1)) * sizeof(T);
  if (int e = allow_smem(k_dg_cell<ND, NQ, T>, sm_cell)) return e;
  k_dg_cell<ND, NQ, T><<<unsigned(c.ntiles), kT, sm_cell, st>>>(metric, tab + L.E, tab + L.w, u, y, c.nc);
  TETMF_LAUNCH_CK();
  const size_t sm_face = (size_t(4) * NQF * ND * 4 + NQF) * sizeof(T) + 6 * NQF * sizeof(int);
  if (c.nfi > 0) {
    if (int e = allow_smem(k_dg_face_interior<ND, NQF, T>, sm_face)) return e;
    k_dg_face_interior<ND, NQF, T><<<unsigned((c.nfi + kT - 1) / kT), kT, sm_face, st>>>(
        c.d_fi_cell, c.d_fi_code, fgi, tab + L.Vf, tab + L.Ef, tab + L.wf, c.d_fperm, u, y, c.nfi);
    TETMF_LAUNCH_CK();
  }
  if (c.nfb > 0) {
    if (int e = allow_smem(k_dg_face_boundary<ND, NQF, T>, sm_face)) return e;
    k_dg_face_boundary<ND, NQF, T><<<unsigned((c.nfb + kT - 1) / kT), kT, sm_face, st>>>(
        c.d_fb_cell, c.d_fb_code, fgb, tab + L.Vf, tab + L.Ef, tab + L.wf, c.d_fperm, u, y, c.nfb);
    TETMF_LAUNCH_CK();
  }
  return FEM_OK;
}


}  // namespace

int dg_apply(Ctx& c, int prec, const void* u, void* y, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64) {
    TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_dg<ND, NQ, NQF, double>(c, static_cast<const double*>(u), static_cast<double*>(y),
                                                           c.d_metric64, c.d_tab64, c.d_fi_geo64, c.d_fb_geo64, st)))
  }
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_dg<ND, NQ, NQF, float>(c, static_cast<const float*>(u), static_cast<float*>(y),
                                                        c.d_metric32, c.d_tab32, c.d_fi_geo32, c.d_fb_geo32, st)))
}


}  // namespace tetmf
