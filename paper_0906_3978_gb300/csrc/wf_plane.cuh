// wf_plane.cuh -- the middle of the Wiener matvec (Sec. 3.3.1: the data term R^T N^-1 R applied
// between the inverse and forward transforms of the signal) on one x-plane at a time, held in
// the distributed shared memory of a thread-block cluster:
//
//     T(x, ., .)  ->  IFFT_y  ->  C2R_z  ->  times D(x, y, z)  ->  R2C_z  ->  FFT_y  ->  T(x, ., .)
//
// It replaces the y pass, z turn and y pass of the separate-kernel form, so an x-plane makes one
// HBM round trip (read T and D, write T: 3 spectrum-sized streams instead of 7).
//
// A plane is N rows (y) by H = N/2 packed kz columns.  The CS CTAs of a cluster split it:
//   phase A / E  CTA c holds kz columns [c KC, c KC + KC) of every row (KC = H / CS) and runs
//                the y transforms of those columns;
//   phase C      CTA c holds rows [c RB, c RB + RB) (RB = N / CS = 2 KC) of every kz column and
//                runs the z transforms of those rows.
// Between them the cluster transposes blocks of RB x KC elements through distributed shared
// memory: block s (rows [s RB, s RB + RB)) of CTA c goes to block c of CTA s.
//
// Shared-memory layout: one tile of N x KC elements, row-major, element (row, col) at
// row * KC + (col ^ (row & (KC - 1))).  The XOR swizzle makes both access patterns free of bank
// conflicts: the y transforms touch one row across the columns, the z transforms one column
// across consecutive rows.  Because RB is a multiple of KC, a block has the same swizzle in the
// CTA that sends it and the CTA that receives it, so the transpose copies raw 16-byte vectors.
#pragma once
#include <cooperative_groups.h>

#include "wf_spectral.cuh"

namespace wf {

// Cluster size for the plane kernel (0: the size runs the separate y / z / y passes).  Needs
// KC = N / (2 CS) in {16, 32} for the swizzle, a portable cluster size (<= 8) and a tile that
// fits one CTA.
template <class R, int N> constexpr int plane_cs() {
  if constexpr (sizeof(cx<R>) != 8) return 0;  // FP32 spectra only
  else return N == 512 ? 8 : N == 384 ? 6 : N == 256 ? 4 : N == 192 ? 3 : N == 128 ? 2 : 0;
}

// Elements per thread (16 or 32): the CTA has N KC / E threads.
template <class R, int N> constexpr int plane_e() { return 16; }

template <class R, int N, int CS, int E>
struct PlaneG {
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  static constexpr int NN = N, H = N / 2, KC = H / CS, RB = N / CS;
  static_assert(CS >= 1 && H % CS == 0 && (KC == 16 || KC == 32) && RB == 2 * KC, "plane geometry");
  static constexpr int NT = N * KC / E;            // E elements per thread in both phases
  static constexpr int TPLY = NT / KC;             // threads per y line (a kz column)
  static constexpr int TPLZ = NT / RB;             // threads per z line (a y row)
  static_assert(NT % KC == 0 && NT % RB == 0 && NT % 32 == 0 && NT <= 1024, "plane threads");
  static constexpr int VE = 16 / (int)sizeof(ST);  // elements per 16-byte vector
  static constexpr int TILE = N * KC;              // elements of the tile
  static constexpr size_t SMEM = (size_t)(TILE + 2 * N) * sizeof(cx<R>);
  static constexpr int BV = RB * KC * (int)sizeof(cx<R>) / 16;  // 16-byte vectors per block
  static constexpr int RMZ = rmax_for(H, TPLZ);  // largest radix of the z transforms
};

// y line `l` (a kz column), element i = row
template <int KC> struct YMap {
  int l;
  WF_D int operator()(int i) const { return i * KC + (l ^ (i & (KC - 1))); }
};
// z line `yl` (a row of this CTA's block), element i = kz
template <int KC, int RB> struct ZMap {
  int yl, s;
  WF_D int operator()(int i) const { return ((i / KC) * RB + yl) * KC + ((i % KC) ^ s); }
};

// 16-byte vector `q` of tile row `row` (elements q VE .. q VE + VE - 1) <-> register vector.
// With two elements per vector the swizzled pair stays aligned; an odd key swaps its halves.
template <class G, class R>
WF_D void tile_put(cx<R>* tile, int row, int q, const float4& v) {
  const int key = row & (G::KC - 1);
  if constexpr (G::VE == 2) {
    float4* p = reinterpret_cast<float4*>(tile + row * G::KC + ((2 * q) ^ (key & ~1)));
    *p = (key & 1) ? make_float4(v.z, v.w, v.x, v.y) : v;
  } else {
    *reinterpret_cast<float4*>(tile + row * G::KC + (q ^ key)) = v;
  }
}
template <class G, class R>
WF_D float4 tile_get(const cx<R>* tile, int row, int q) {
  const int key = row & (G::KC - 1);
  if constexpr (G::VE == 2) {
    const float4 v = *reinterpret_cast<const float4*>(tile + row * G::KC + ((2 * q) ^ (key & ~1)));
    return (key & 1) ? make_float4(v.z, v.w, v.x, v.y) : v;
  } else {
    return *reinterpret_cast<const float4*>(tile + row * G::KC + (q ^ key));
  }
}

// Columns [kc0, kc0 + KC) of the N rows of a plane (row stride H) <-> tile.
template <class G, class R>
WF_D void plane_load(cx<R>* tile, const typename G::ST* g, int tid) {
  constexpr int VPR = G::KC / G::VE, NV = G::NN * VPR, PER = NV / G::NT;
  static_assert(NV % G::NT == 0, "plane load");
  float4 buf[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * G::NT;
    buf[k] = *reinterpret_cast<const float4*>(g + (size_t)(idx / VPR) * G::H + (idx % VPR) * G::VE);
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * G::NT;
    tile_put<G>(tile, idx / VPR, idx % VPR, buf[k]);
  }
}
template <class G, class R>
WF_D void plane_store(const cx<R>* tile, typename G::ST* g, int tid) {
  constexpr int VPR = G::KC / G::VE, NV = G::NN * VPR, PER = NV / G::NT;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * G::NT;
    *reinterpret_cast<float4*>(g + (size_t)(idx / VPR) * G::H + (idx % VPR) * G::VE) = tile_get<G>(tile, idx / VPR, idx % VPR);
  }
}

// Cluster transpose: block s of this CTA (c) -> block c of CTA s, for every s != c.  All
// outgoing blocks are read into registers, the cluster synchronises (every block except the
// diagonal one is then free), the blocks are written into the peers' shared memory, and the
// cluster synchronises again so that the incoming blocks are visible.
template <class G, int CS, class R>
WF_D void plane_transpose(cx<R>* tile, cooperative_groups::cluster_group& cl, int c, int tid) {
  constexpr int TOT = (CS - 1) * G::BV, PER = (TOT + G::NT - 1) / G::NT;
  float4* loc = reinterpret_cast<float4*>(tile);
  float4 buf[PER];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * G::NT;
    if (TOT % G::NT == 0 || idx < TOT) {
      int s = c + 1 + idx / G::BV;
      if (s >= CS) s -= CS;
      buf[k] = loc[s * G::BV + idx % G::BV];
    }
  }
  cl.sync();
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * G::NT;
    if (TOT % G::NT == 0 || idx < TOT) {
      int s = c + 1 + idx / G::BV;
      if (s >= CS) s -= CS;
      float4* peer = cl.map_shared_rank(loc, (unsigned)s);
      peer[c * G::BV + idx % G::BV] = buf[k];
    }
  }
  cl.sync();
}

// z phase: the RB rows of this CTA (global rows y0 + yl): C2R, times D, R2C.  Returns this
// thread's share of sum D T^2 over the real samples T (the data term of <p, A p>).
template <class G, class R, int N>
WF_D double plane_zturn(cx<R>* tile, const typename G::SS* __restrict__ Drow0, const cx<R>* tw, int tid) {
  using SS = typename G::SS;
  constexpr int H = G::H, KC = G::KC, RB = G::RB, TPLZ = G::TPLZ;
  const int yl = tid % RB, t = tid / RB;
  const ZMap<KC, RB> map{yl, yl & (KC - 1)};
  c2r_prep_map<R, N>(tile, map, t, TPLZ, tw);
  __syncthreads();
  fft_line_map<R, H, TPLZ, +1, 4, G::RMZ>(tile, map, t, tw);
  // element m of row yl holds the real samples z = 2m, 2m + 1: multiply by D, a 16-byte vector
  // of D (16 / sizeof(SS) reals = VE elements) at a time, rows read whole
  constexpr int DPR = H / G::VE, ND = RB * DPR, PER = ND / G::NT;
  static_assert(ND % G::NT == 0, "plane D");
  float4 dv[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * G::NT;
    dv[k] = *reinterpret_cast<const float4*>(Drow0 + (size_t)(idx / DPR) * N + 2 * G::VE * (idx % DPR));
  }
  typename AccFor<SS>::T acc;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * G::NT;
    const int r = idx / DPR, m = G::VE * (idx % DPR);
    const int row = (m / KC) * RB + r, q = (m % KC) / G::VE;
    const float4 v = tile_get<G>(tile, row, q);
    float4 o;
    if constexpr (G::VE == 2) {
      o = make_float4(v.x * dv[k].x, v.y * dv[k].y, v.z * dv[k].z, v.w * dv[k].w);
      acc.add_prod(o.x, v.x);
      acc.add_prod(o.y, v.y);
      acc.add_prod(o.z, v.z);
      acc.add_prod(o.w, v.w);
    } else {
      const double2 e = *reinterpret_cast<const double2*>(&v);
      const double2 d = *reinterpret_cast<const double2*>(&dv[k]);
      const double2 p = make_double2(e.x * d.x, e.y * d.y);
      acc.add_prod(p.x, e.x);
      acc.add_prod(p.y, e.y);
      o = *reinterpret_cast<const float4*>(&p);
    }
    tile_put<G>(tile, row, q, o);
  }
  __syncthreads();
  fft_line_map<R, H, TPLZ, -1, 4, G::RMZ>(tile, map, t, tw);
  r2c_post_map<R, N>(tile, map, t, TPLZ, tw);
  return acc.get();
}

// One x-plane per cluster: grid (N CS, 1, systems), cluster (CS, 1, 1) (set at launch), block G::NT.
// D = nbar w / V_c (it carries the 1/V_c of the inverse transform).  In place on `spec`.
// partials[blockIdx.x] (per system) receives the CTA's sum of D T^2, as the z turn's do.
template <class R, int N, int CS, int E, int MINB = 1>
__global__ void __launch_bounds__(PlaneG<R, N, CS, E>::NT, MINB)
k_plane_turn(typename Store<R>::T* __restrict__ spec, const typename Store<R>::S* __restrict__ D,
             const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials, const CgScal* __restrict__ sc,
             Bat bt) {
  using G = PlaneG<R, N, CS, E>;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::TILE;
  __shared__ double red[32];
  const int z = blockIdx.z;
  if (sc && sc[z].done) return;  // the whole cluster belongs to system z: it leaves together
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int x = blockIdx.x / CS;
  const int tid = threadIdx.x;
  typename G::ST* plane = spec + z * bt.spec + (size_t)x * N * G::H;
  const typename G::SS* Drow0 = D + z * bt.real + ((size_t)x * N + (size_t)c * G::RB) * N;
  // the D rows of phase C go to L2 now, while the plane is transformed along y
  if (tid < G::RB) prefetch_l2(Drow0 + (size_t)tid * N, (unsigned)(N * sizeof(typename G::SS)));
  for (int e = tid; e < 2 * N; e += G::NT) tw[e] = ld_c<R>(twtab + e);
  // phase A: columns [c KC, c KC + KC), inverse transform along y (W_N^e = tw[2 e])
  plane_load<G>(tile, plane + c * G::KC, tid);
  __syncthreads();
  fft_line_map<R, N, G::TPLY, +1, 2>(tile, YMap<G::KC>{tid % G::KC}, tid / G::KC, tw);
  // phase B: to rows; C: z turn; D: back to columns
  plane_transpose<G, CS>(tile, cl, c, tid);
  const double dsum = plane_zturn<G, R, N>(tile, Drow0, tw, tid);
  plane_transpose<G, CS>(tile, cl, c, tid);
  // phase E: forward transform along y, store
  fft_line_map<R, N, G::TPLY, -1, 2>(tile, YMap<G::KC>{tid % G::KC}, tid / G::KC, tw);
  plane_store<G>(tile, plane + c * G::KC, tid);
  const double sum = block_sum(dsum, red);
  if (tid == 0) partials[z * bt.part + blockIdx.x] = sum;
}

// Launch k_plane_turn over nb systems on stream st with the cluster shape (CS, 1, 1).  The
// caller has raised the kernel's dynamic shared-memory limit to PlaneG::SMEM.
template <class R, int N, int CS, int E, int MINB = 1>
static cudaError_t plane_turn_launch(typename Store<R>::T* spec, const typename Store<R>::S* D,
                                     const typename Store<R>::T* tw,
                                     double* partials, const CgScal* sc, Bat bt, int nb, cudaStream_t st) {
  using G = PlaneG<R, N, CS, E>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(N * CS, 1, nb);
  cfg.blockDim = dim3(G::NT, 1, 1);
  cfg.dynamicSmemBytes = G::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_plane_turn<R, N, CS, E, MINB>, spec, D, tw, partials, sc, bt);
}

}  // namespace wf
