// Cluster-resident PCG for small systems (Sec. 4 PCG with the two-level
// preconditioner of Algorithm 1): one thread-block cluster of C <= 16 CTAs
// (one per SM) keeps every vector of the solve and its rows of P in shared
// memory for the whole solve.  Rank q of the cluster owns nodes
// [q nl, (q + 1) nl) and copies its rows of A once into shared memory as a
// rank-local ELL block (entry j of local row i at j nlp + i: the value and a
// reference to the neighbour, owner rank and index within the owner, resolved
// once), together with D^-1 and A_c^-1; after that an iteration reads only
// shared memory, its own and, for neighbours owned by another rank, the
// owner's through distributed shared memory (generic addresses of the
// cluster's shared-memory window).  Global memory is not touched inside the
// loop: every cluster barrier acquires at cluster scope, which would send
// cached global reads back to L2 in every phase.  The phases of an iteration
// are separated by the cluster's hardware barrier instead of a grid barrier
// through L2.  Scalars
// (p^T q, r^T r, r^T z) and the coarse right-hand side P^T rho are added up by
// every rank from all ranks' partials in rank order, so all ranks take
// identical decisions (stop, breakdown, maxit) and pass the same sequence of
// cluster barriers; no rank leaves before a final barrier, so no rank reads
// the shared memory of one that has exited.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace {

namespace cgx = cooperative_groups;

constexpr int CT = 512;     // threads per CTA of the cluster solver
constexpr int CL_MAX = 16;  // CTAs per cluster (non-portable size 16)

struct ClusterArgs {
  int64_t n;
  int nl;    // nodes per rank
  int nlp;   // leading dimension of the local P block (odd: conflict-free columns)
  int k, r;  // stored / active rank
  int nu1, nu2, flexible, maxit;
  double tol;
  const double* b;
  double* x;
  const void* P;     // tiled P (precision T), k columns
  const void* Ainv;  // A_c^-1, r x r column-major (precision T)
  int ew;            // ELL width: most off-diagonal entries of a row
  int rg;            // threads per column of the restriction (power of two <= 32)
  int lc;            // lanes per column of the coarse solve (power of two <= 16)
  int ainv_smem;     // A_c^-1 is copied into shared memory
  PcgState* st;
  unsigned long long* ptimes;  // optional: rank 0's time between marks, ns (slots 14 + mark)
};

// Off-diagonal entries per row of the stencil kinds (the sparse kind takes
// the operator's widest row).
template <int KIND>
__host__ __device__ constexpr int cluster_stencil_width() {
  return KIND == ST_5PT ? 4 : KIND == ST_7PT ? 6 : KIND == ST_9PT ? 8 : 0;
}

// Dynamic shared memory of one rank, FP64 arrays first: 5 FP64 vectors (x, r,
// p, q, z), the ELL values and diagonal in FP64 when T is narrower; then in
// precision T 3 vectors (rT, w0, w1), the rank's rows of P (r x nlp), the
// coarse vectors (partial, total, correction: 3 r), the ELL values, diagonal
// and D^-1, A_c^-1 (r x r, when copied); then the ELL references (int).
template <typename T>
__host__ __device__ inline size_t cluster_smem(int nl, int nlp, int r, int ew, bool ainv) {
  const size_t wide = sizeof(T) < sizeof(double) ? (size_t)ew * nlp + nl : 0;
  return ((size_t)5 * nl + wide) * sizeof(double) +
         ((size_t)3 * nl + (size_t)r * nlp + (size_t)3 * r + (size_t)ew * nlp + 2 * (size_t)nl +
          (ainv ? (size_t)r * r : 0)) * sizeof(T) +
         (size_t)ew * nlp * sizeof(int) + 64;
}

// Scalars of the solve, kept in shared memory and updated by thread 0 only:
// GB300 runs FP64 at 1/64 of the FP32 rate, so scalar FP64 work (sums of the
// ranks' partials, alpha, beta, the stop tests) done redundantly by every
// thread of a 512-thread CTA would cost microseconds per step.
struct ClScalars {
  double bnorm2, tol2bn, rz, pq, alpha, beta, rr;
  int iter, status, done, pad;
};

template <int KIND, typename T>
__global__ void __launch_bounds__(CT, 1) k_pcg_cluster(StencilView<double> A64, StencilView<T> AT, T omega,
                                                       ClusterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double slot[8];             // this rank's published partials
  __shared__ double red[CT];              // per-thread partials of a CTA sum
  __shared__ double stot[8];             // cluster totals of the slots (thread 0)
  __shared__ ClScalars cs;
  __shared__ double* rp_x[CL_MAX];       // the ranks' vectors (generic addresses)
  __shared__ double* rp_p[CL_MAX];
  __shared__ double* rp_z[CL_MAX];
  __shared__ T* rp_w0[CL_MAX];
  __shared__ T* rp_w1[CL_MAX];
  __shared__ T* rp_c[CL_MAX];
  __shared__ double* rp_slot[CL_MAX];
  cgx::cluster_group cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks();
  const int tid = threadIdx.x;
  const int nl = a.nl, nlp = a.nlp, r = a.r;
  constexpr int EW = cluster_stencil_width<KIND>();
  const int ew = EW ? EW : a.ew;
  constexpr bool narrow = sizeof(T) < sizeof(double);
  const int lo = rank * nl;
  const int cnt = max(0, min((int)a.n, lo + nl) - lo);
  double* xv = reinterpret_cast<double*>(smem_raw);
  double* rv = xv + nl;
  double* pv = rv + nl;
  double* qv = pv + nl;
  double* zv = qv + nl;
  double* e64 = zv + nl;               // ELL values in FP64 (narrow T only)
  double* d64 = e64 + (narrow ? (size_t)ew * nlp : 0);
  T* rT = reinterpret_cast<T*>(d64 + (narrow ? nl : 0));
  T* w0 = rT + nl;
  T* w1 = w0 + nl;
  T* Pl = w1 + nl;           // Pl[j * nlp + i]
  T* cpart = Pl + (size_t)r * nlp;
  T* ctot = cpart + r;
  T* ev = ctot + r;
  T* eT = ev + r;            // ELL values in T: eT[j * nlp + i]
  T* dT = eT + (size_t)ew * nlp;
  T* diT = dT + nl;          // D^-1
  T* As = diT + nl;          // A_c^-1 (column-major), when copied
  int* eref = reinterpret_cast<int*>(As + (a.ainv_smem ? (size_t)r * r : 0));
  if (!narrow) {  // FP64 preconditioner: one copy of the values serves both
    e64 = reinterpret_cast<double*>(eT);
    d64 = reinterpret_cast<double*>(dT);
  }
  if (tid < C) {
    rp_x[tid] = cl.map_shared_rank(xv, tid);
    rp_p[tid] = cl.map_shared_rank(pv, tid);
    rp_z[tid] = cl.map_shared_rank(zv, tid);
    rp_w0[tid] = cl.map_shared_rank(w0, tid);
    rp_w1[tid] = cl.map_shared_rank(w1, tid);
    rp_c[tid] = cl.map_shared_rank(cpart, tid);
    rp_slot[tid] = cl.map_shared_rank(&slot[0], tid);
  }
  // (A v)_i of local row i from the ELL block: values `val`, diagonal `dg`,
  // this rank's vector `own`, the ranks' vectors `rem` (own rows straight
  // from this rank's shared memory)
  auto ell = [&](auto* own, auto* const* rem, const auto* val, const auto* dg, int i) {
    auto s = dg[i] * own[i];
#pragma unroll 4
    for (int j = 0; j < ew; ++j) {
      const int rf = eref[j * nlp + i];
      const int o = rf >> 16;
      const auto* bp = o == rank ? own : rem[o];
      s += val[j * nlp + i] * bp[rf & 0xffff];
    }
    return s;
  };
  // Cross-rank totals of the slots in `mask` into stot: warp sl reads slot
  // sl of rank q in lane q (remote reads in parallel) and adds them by a
  // shuffle tree (a fixed order, identical on every rank; few dependent FP64
  // adds, which GB300 executes with a long latency).  Called by every thread
  // right after a cluster barrier; ends with a CTA barrier.
  auto gather = [&](unsigned mask) {
    const int w = tid >> 5, lane = tid & 31;
    if (w < 8 && ((mask >> w) & 1u)) {
      double v = lane < C ? rp_slot[lane][w] : 0.0;
      v = warp_sum(v);
      if (lane == 0) stot[w] = v;
    }
    __syncthreads();
  };
  // this rank's partial of a sum over its nodes into slot `sl`: every thread
  // stores its value, warp 0 adds the values of the warps that hold rows
  // column by column and then its 32 lane sums by a shuffle tree.  One FP64
  // add per value instead of the five of a shuffle tree in every warp: GB300
  // executes FP64 at 1/64 of the FP32 rate, and threads without rows hold 0.
  const int nact = (min(cnt, CT) + 31) >> 5;
  auto partial = [&](double v, int sl) {
    __syncthreads();  // red is free again
    red[tid] = v;
    __syncthreads();
    if (tid < 32) {
      double t = red[tid];
      for (int w = 1; w < nact; ++w) t += red[w * 32 + tid];
      t = warp_sum(t);
      if (tid == 0) slot[sl] = t;
    }
  };
  // phase marks (NLSP_PHASE_TIMERS=1): time since the previous mark, rank 0
  const bool timed = a.ptimes && rank == 0 && tid == 0;
  unsigned long long t_last = 0, tacc[13];
  for (int q = 0; q < 13; ++q) tacc[q] = 0;
  if (timed) t_last = tma::now_ns();
  auto mark = [&](int id) {  // accumulated in registers, written once at the end
    if (timed) {
      const unsigned long long t = tma::now_ns();
      tacc[id] += t - t_last;
      t_last = t;
    }
  };
  const T* Pg = reinterpret_cast<const T*>(a.P);
  const T* Ainv = reinterpret_cast<const T*>(a.Ainv);
  double bb = 0.0;
  for (int i = tid; i < cnt; i += CT) {
    const double bi = a.b[lo + i];
    rv[i] = bi;
    xv[i] = 0.0;
    pv[i] = 0.0;
    qv[i] = 0.0;
    zv[i] = 0.0;
    rT[i] = (T)bi;
    bb += bi * bi;
  }
  for (int e = tid; e < r * cnt; e += CT) {
    const int j = e / cnt, i = e - j * cnt;
    Pl[j * nlp + i] = Pg[tiled_index(lo + i, j, a.k)];
  }
  if (a.ainv_smem)
    for (int e = tid; e < r * r; e += CT) As[e] = Ainv[e];
  // the rank's rows as an ELL block: neighbours in the order the operator
  // visits them, then (own row, 0) up to the width
  for (int i = tid; i < cnt; i += CT) {
    const int64_t g = lo + i;
    int j = 0;
    for_each_neighbour<KIND>(AT, g, node_coord<KIND>(g, AT.N), [&](int64_t m, NodeCoord, T v) {
      if (j < ew) {
        const int o = (int)(m / nl);
        eref[j * nlp + i] = (o << 16) | (int)(m - (int64_t)o * nl);
        eT[j * nlp + i] = v;
      }
      ++j;
    });
    for (; j < ew; ++j) {
      eref[j * nlp + i] = (rank << 16) | i;
      eT[j * nlp + i] = T(0);
    }
    dT[i] = stencil_diag<KIND>(AT, g);
    diT[i] = stencil_dinv<KIND>(AT, g);
    if (narrow) {
      int j2 = 0;
      for_each_neighbour<KIND>(A64, g, node_coord<KIND>(g, A64.N), [&](int64_t, NodeCoord, double v) {
        if (j2 < ew) e64[j2 * nlp + i] = v;
        ++j2;
      });
      for (; j2 < ew; ++j2) e64[j2 * nlp + i] = 0.0;
      d64[i] = stencil_diag<KIND>(A64, g);
    }
  }
  const T* Ac = a.ainv_smem ? As : Ainv;
  partial(bb, 4);
  cl.sync();
  gather(1u << 4);
  if (tid == 0) {
    const double bn = stot[4];
    cs.bnorm2 = bn;
    cs.tol2bn = a.tol * a.tol * bn;
    cs.rz = cs.pq = cs.alpha = cs.beta = 0.0;
    cs.rr = bn;
    cs.iter = 0;
    cs.status = NLSP_OK;
    cs.done = 0;
    if (!isfinite(bn)) {  // a non-finite right-hand side
      cs.status = NLSP_ERR_BREAKDOWN;
      cs.done = 1;
    } else if (!(bn > 0.0)) {  // b = 0: x = 0 after no iteration
      cs.done = 1;
      cs.rr = 0.0;
    }
  }
  __syncthreads();

  // z = B r, from the first sweep w0 = omega D^-1 rT (local); writes z (FP64)
  // and publishes r^T z (slot 2) and r^T z_old (slot 3)
  auto precondition = [&]() {
    T* cur = w0;
    T* oth = w1;
    T* const* rc = rp_w0;
    T* const* ro = rp_w1;
    for (int sw = 1; sw < a.nu1; ++sw) {
      cl.sync();
      for (int i = tid; i < cnt; i += CT) {
        const T az = ell(cur, rc, eT, dT, i);
        oth[i] = cur[i] + omega * diT[i] * (rT[i] - az);
      }
      T* t = cur; cur = oth; oth = t;
      T* const* tt = rc; rc = ro; ro = tt;
    }
    mark(3);
    cl.sync();
    mark(4);
    // rho = rT - A cur into oth (nobody reads oth in this phase)
    for (int i = tid; i < cnt; i += CT) {
      oth[i] = rT[i] - ell(cur, rc, eT, dT, i);
    }
    __syncthreads();
    mark(5);
    // restriction partial: c_j = sum over the rank's nodes of P_ij rho_i, rg
    // threads per column (rg a power of two <= 32, so a column's threads are
    // lanes of one warp)
    const int rg = a.rg;
    for (int base = 0; base < rg * r; base += CT) {  // uniform trip count: whole warps shuffle
      const int jj = base + tid;
      const int j = jj / rg, part = jj & (rg - 1);
      T s = T(0);
      if (j < r)
        for (int i = part; i < cnt; i += rg) s += Pl[j * nlp + i] * oth[i];
      for (int off = rg >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (part == 0 && j < r) cpart[j] = s;
    }
    mark(6);
    cl.sync();
    mark(7);
    // c = sum of the ranks' partials and e = A_c^-1 c, lc lanes per column
    // (lc a power of two <= 16; each lane adds the ranks q, q + lc, ... and
    // the rows q, q + lc, ... of A_c^-1, then a shuffle tree over the lanes,
    // in the same order on every rank)
    const int lc = a.lc;
    for (int base = 0; base < lc * r; base += CT) {  // uniform trip count: whole warps shuffle
      const int jj = base + tid;
      const int j = jj / lc, q = jj & (lc - 1);
      T v = T(0);
      if (j < r)
#pragma unroll 4
        for (int o = q; o < C; o += lc) v += rp_c[o][j];
      for (int off = lc >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (q == 0 && j < r) ctot[j] = v;
    }
    __syncthreads();
    for (int base = 0; base < lc * r; base += CT) {
      const int jj = base + tid;
      const int j = jj / lc, q = jj & (lc - 1);
      T v = T(0);
      if (j < r)
        for (int l = q; l < r; l += lc) v += Ac[(int64_t)l * r + j] * ctot[l];
      for (int off = lc >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (q == 0 && j < r) ev[j] = v;
    }
    __syncthreads();
    mark(8);
    // prolongation: cur += P e
    for (int i = tid; i < cnt; i += CT) {
      T s = T(0);
      for (int j = 0; j < r; ++j) s += Pl[j * nlp + i] * ev[j];
      cur[i] += s;
    }
    mark(9);
    // post-smoothing; the last sweep writes z in FP64 with r^T z, r^T z_old
    double pz = 0.0, pzo = 0.0;
    for (int sw = 1; sw <= a.nu2; ++sw) {
      cl.sync();
      const bool last = sw == a.nu2;
      for (int i = tid; i < cnt; i += CT) {
        const T az = ell(cur, rc, eT, dT, i);
        const T v = cur[i] + omega * diT[i] * (rT[i] - az);
        if (last) {
          const double zn = (double)v;
          pzo += rv[i] * zv[i];
          pz += rv[i] * zn;
          zv[i] = zn;
        } else {
          oth[i] = v;
        }
      }
      if (!last) {
        T* t = cur; cur = oth; oth = t;
        T* const* tt = rc; rc = ro; ro = tt;
      }
    }
    partial(pz, 2);
    partial(pzo, 3);
    mark(10);
  };

  // q = A z + beta q, p = z + beta p, publishes p^T q (slot 0)
  auto direction = [&](double bt) {
    double s = 0.0;
    for (int i = tid; i < cnt; i += CT) {
      const double az = ell(zv, rp_z, e64, d64, i);
      const double pn = zv[i] + bt * pv[i];
      const double qn = az + bt * qv[i];
      pv[i] = pn;
      qv[i] = qn;
      s += pn * qn;
    }
    partial(s, 0);
  };

  if (!cs.done) {
    for (int i = tid; i < cnt; i += CT) w0[i] = omega * diT[i] * rT[i];
    precondition();
    cl.sync();
    gather(1u << 2);
    if (tid == 0) {
      const double rz = stot[2];
      if (!(rz > 0.0) || !isfinite(rz)) {
        cs.status = NLSP_ERR_BREAKDOWN;
        cs.done = 1;
      }
      cs.rz = rz;
    }
    __syncthreads();
    if (!cs.done) direction(0.0);
  }
  while (!cs.done && cs.iter < a.maxit) {
    cl.sync();  // S1: p^T q
    gather(1u << 0);
    mark(0);
    if (tid == 0) {
      const double pq = stot[0];
      cs.pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        cs.status = NLSP_ERR_BREAKDOWN;
        cs.done = 1;
      } else {
        cs.alpha = cs.rz / pq;
      }
    }
    __syncthreads();
    if (cs.done) break;
    const double alpha = cs.alpha;
    double s = 0.0;
    for (int i = tid; i < cnt; i += CT) {
      const double xi = xv[i] + alpha * pv[i];
      const double ri = rv[i] - alpha * qv[i];
      xv[i] = xi;
      rv[i] = ri;
      const T rt = (T)ri;
      rT[i] = rt;
      w0[i] = omega * diT[i] * rt;
      s += ri * ri;
    }
    partial(s, 1);
    if (tid == 0) cs.iter += 1;
    mark(1);
    cl.sync();  // S2: r^T r
    gather(1u << 1);
    mark(2);
    if (tid == 0) {
      const double rr = stot[1];
      cs.rr = rr;
      if (!isfinite(rr)) {
        cs.status = NLSP_ERR_BREAKDOWN;
        cs.done = 1;
      } else if (rr <= cs.tol2bn) {
        cs.done = 1;
      }
    }
    __syncthreads();
    if (cs.done || cs.iter >= a.maxit) break;
    precondition();
    cl.sync();  // r^T z
    gather((1u << 2) | (1u << 3));
    mark(11);
    if (tid == 0) {
      const double rzn = stot[2], rzo = stot[3];
      if (!(rzn > 0.0) || !isfinite(rzn)) {
        cs.status = NLSP_ERR_BREAKDOWN;
        cs.done = 1;
      } else {
        cs.beta = a.flexible ? (rzn - rzo) / cs.rz : rzn / cs.rz;
        cs.rz = rzn;
      }
    }
    __syncthreads();
    if (cs.done) break;
    direction(cs.beta);
    mark(12);
  }
  // true residual ||b - A x||^2 (x of every rank is visible after a barrier)
  cl.sync();
  double tr = 0.0;
  for (int i = tid; i < cnt; i += CT) {
    const double d = a.b[lo + i] - ell(xv, rp_x, e64, d64, i);
    tr += d * d;
  }
  partial(tr, 5);
  for (int i = tid; i < cnt; i += CT) a.x[lo + i] = xv[i];
  cl.sync();
  gather(1u << 5);
  if (rank == 0 && tid == 0) {
    PcgState* st = a.st;
    st->bnorm2 = cs.bnorm2;
    st->tol2bn = cs.tol2bn;
    st->rz = cs.rz;
    st->pq = cs.pq;
    st->alpha = cs.alpha;
    st->beta = cs.beta;
    st->rr = cs.rr;
    st->true_rr = stot[5];
    st->iter = cs.iter;
    st->done = cs.done;
    st->status = cs.status;
    st->maxit = a.maxit;
    st->flexible = a.flexible;
  }
  if (timed)
    for (int q = 0; q < 13; ++q) a.ptimes[14 + q] += tacc[q];
  cl.sync();  // no rank leaves while another may still read its shared memory
}

}  // namespace
