// k_sweepg.cu -- the source iteration of Algorithm 1 step 4 for
// mixed-precision DLR instances, with the r collocation angles swept in
// groups of kGA angles of one quadrant per warp:
//   Om^(j).grad psi_j + (sigma + 1/(c dt)) psi_j
//       = sigma_s/(4 pi) gamma^T Psi + q + psi0_j / (c dt)
// (Eq. steady state collocation of Haut et al., phi = beta^T What^{-1} Psi =
// gamma^T Psi with gamma = What^{-T} beta), DG0 upwind cells.
//
// Organisation (one loop of kernels per step for every instance of a batch,
// see the section "The source iteration as a loop of kernels" below):
//   * a warp sweeps one band of 32 rows for the kGA angles of its group at
//     once (lane i = row i, anti-diagonal wavefront: lane i reaches column u
//     at step t = u + i; the lower neighbour comes from lane i - 1 by a
//     shuffle, the left one stays in a register), so each step carries kGA
//     independent recurrences;
//   * its inputs (the angles' fixed sources, sigma_t and sigma_s phi / 4 pi)
//     are stored in the skewed band layout of grp_off, where one
//     (band, 32-step window) block is 4 KB contiguous: a warp streams them
//     into shared memory with bulk asynchronous copies (cp.async.bulk, one
//     mbarrier per stage; the fixed sources with an L2 evict-first policy)
//     and reads 4 steps per lane with one conflict-free 16-byte load;
//   * instead of psi the sweep writes, per group, sum_j gamma_j psi_j in the
//     same skewed layout (in place of the stage's sigma_s phi values, then
//     one bulk store per window); the scalar-flux kernels sum the groups'
//     partials per quadrant, then the four quadrant sums per cell;
//   * psi itself is written only once, by one more sweep after the source
//     iteration has stopped, with the sigma_s phi of the last iteration
//     (the same inputs and arithmetic, so the same psi bit for bit);
//   * the band's top row goes to the next band through a shared-memory edge
//     row behind a progress counter (bands of one CTA) or tagged 64-bit
//     words in global memory (bands of different CTAs), as in k_sweep.cu.
// Every wait is bounded in time and leaves on the launch's abort flag.
#include "dlr_internal.cuh"

namespace dlr {

namespace {

constexpr int kNWg = 4;                  // sweeping warps per CTA (one band each at a time)
constexpr int kSubG = 16;                // progress granularity (steps)
constexpr int kEdgePadG = 32;            // edge row padding (columns -31 .. -1)
constexpr uint64_t kWaitNsG = 4000000000ull;
constexpr unsigned kFullG = 0xffffffffu;
constexpr int kBlk = 1024;               // floats per (band, window) block

__host__ __device__ inline int edge_ld_g(int nx_max) { return (nx_max + 3) / 4 * 4 + 128; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 4 KB from global to shared memory, completing on the mbarrier (bulk
// asynchronous copy; both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(m))
      : "memory");
}
// The same with an L2 eviction-priority policy (createpolicy).
__device__ __forceinline__ void bulk_load_hint(void *dst, const void *src, unsigned bytes, uint64_t *m,
                                               uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(m)), "l"(policy)
      : "memory");
}
// L2 policies: the fixed sources stream through L2 (read once per
// iteration, 8 x the partials' bytes), the partials and sigma_s phi stay
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 4 KB from shared to global memory (bulk asynchronous copy, tracked by the
// issuing thread's bulk group)
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes, uint64_t policy) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes), "l"(policy)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the issuing thread's bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// ... and have completed (their writes are performed)
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// orders this thread's earlier generic shared-memory accesses before later
// asynchronous-proxy writes to the same memory (a stage is reused)
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ unsigned long long ld_relaxed_g(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_g(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v));
}

__device__ __forceinline__ float f4c(const float4 &v, int s) {
  return s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w;
}
__device__ __forceinline__ void f4s(float4 &v, int s, float x) {
  if (s == 0) v.x = x; else if (s == 1) v.y = x; else if (s == 2) v.z = x; else v.w = x;
}

// Bounded wait of lane 0 until *flag >= need (progress of the band below).
// Each warp of the sweep has its scheduler to itself (four warps per CTA,
// one CTA per SM), so the poll spins without sleeping: a sleeping waiter
// wakes late, and every band below the last adds its delay to the lag of
// the bands above it.
__device__ __forceinline__ bool wait_flag(volatile int *flag, int need, volatile int *abort_flag) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) {
    if (*flag < need) {
      const uint64_t t0 = global_ns();
      unsigned spins = 0;
      while (*flag < need) {
        if ((++spins & 255u) == 0) {
          if (*abort_flag || global_ns() - t0 > kWaitNsG) { ok = false; break; }
        }
      }
    }
    __threadfence_block();
  }
  ok = __shfl_sync(kFullG, ok, 0);
  __syncwarp();
  return ok;
}

// Bounded wait for a stage's bulk copies (all lanes).
__device__ __forceinline__ bool wait_stage(uint64_t *m, unsigned parity, volatile int *abort_flag) {
  if (mbar_try_wait(m, parity)) return true;
  const uint64_t t0 = global_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(m, parity)) {
    if ((++spins & 15u) == 0) {
      bool stop = false;
      if ((threadIdx.x & 31) == 0) stop = *abort_flag || global_ns() - t0 > kWaitNsG;
      if (__shfl_sync(kFullG, stop, 0)) return false;
    }
  }
  return true;
}

// Wait for a stage's copies after a failure elsewhere: bulk copies complete
// by themselves, so this ignores the abort flag (bounded all the same).
__device__ __forceinline__ void drain_stage(uint64_t *m, unsigned parity) {
  const uint64_t t0 = global_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(m, parity)) {
    if ((++spins & 15u) == 0) {
      bool stop = false;
      if ((threadIdx.x & 31) == 0) stop = global_ns() - t0 > kWaitNsG / 4;
      if (__shfl_sync(kFullG, stop, 0)) return;
    }
  }
}

// One group of the sweep: up to G angles of one quadrant of one instance.
template <int G>
struct GrpArgs {
  int nx, ny, nwin, quad, na;
  float ax[G], ay[G], axy[G], gam[G], in_x[G], in_y[G];
  const float *sg;     // the group's blocks of fixed sources and sigma_t (grp_sgk)
  const float *sp;     // skewed sigma_s phi / 4 pi of the quadrant (this sweep's parity)
  float *part;         // the group's partial scalar flux (skewed), or nullptr
  float *psi[G];       // final sweep: the angles' columns of Psi (column-major), else nullptr
};

struct GrpSmem {
  float *stages;   // NW warps x S stages x (G + 2) blocks
  uint64_t *mbar;  // NW x S
  float *edge;     // (NW + 1) rows x G x edge_ld
  int *prog;       // bands_max
  int edge_ld, S;
};

// Per-warp pipeline state: the parity bit of each stage's mbarrier.
struct Pipe {
  unsigned parity;  // bit s: parity of the next completion of stage s
};

// Window k of band b into a stage: the group's fixed sources and sigma_t
// (one contiguous (G + 1) x 4 KB copy) and sigma_s phi / 4 pi (4 KB).
template <int G>
__device__ __forceinline__ void issue_window(const GrpArgs<G> &A, int b, int k, float *stage, uint64_t *m) {
  const size_t bi = (size_t)b * A.nwin + k;
  mbar_expect_tx(m, (G + 2) * kBlk * 4);
  bulk_load_hint(stage, A.sg + bi * (G + 1) * kBlk, (G + 1) * kBlk * 4, m, policy_evict_first());
  bulk_load(stage + (G + 1) * kBlk, A.sp + bi * kBlk, kBlk * 4, m);
}

// The global edge words of one sub-window: lane l < kSubG holds the G words
// of column t0 + l.  Reloaded until every tag matches (bounded in time),
// then decoded into the band's shared edge row.
template <int G>
__device__ __forceinline__ void gedge_load(const unsigned long long *g, int t0, int nx,
                                           unsigned long long (&w)[G]) {
  const int lane = threadIdx.x & 31, c = t0 + lane;
  if (lane < kSubG && c < nx) {
#pragma unroll
    for (int a = 0; a < G; ++a) w[a] = ld_relaxed_g(g + (size_t)c * G + a);
  }
}

template <int G>
__device__ __forceinline__ bool gedge_take(const unsigned long long *g, int t0, int nx, unsigned tag,
                                           unsigned long long (&w)[G], float *edge_in, int ld,
                                           volatile int *abort_flag) {
  const int lane = threadIdx.x & 31;
  const bool mine = lane < kSubG && t0 + lane < nx;
  auto valid = [&]() {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < G; ++a) ok = ok && (unsigned)(w[a] >> 32) == tag;
    return !mine || ok;
  };
  if (!__all_sync(kFullG, valid())) {
    const uint64_t ts = global_ns();
    unsigned spins = 0;
    do {
      gedge_load<G>(g, t0, nx, w);
      if ((++spins & 31u) == 0) {
        bool stop = false;
        if (lane == 0) stop = *abort_flag || global_ns() - ts > kWaitNsG;
        if (__shfl_sync(kFullG, stop, 0)) return false;
      }
    } while (!__all_sync(kFullG, valid()));
  }
  if (mine) {
#pragma unroll
    for (int a = 0; a < G; ++a) edge_in[a * ld + t0 + lane] = __uint_as_float((unsigned)w[a]);
  }
  __syncwarp();
  gedge_load<G>(g, t0 + kSubG, nx, w);
  return true;
}

// Bounded wait until the words of columns t0 .. t0 + kSubG - 1 carry tag.
template <int G>
__device__ __forceinline__ bool gedge_ready(const unsigned long long *g, int t0, int nx, unsigned tag,
                                            volatile int *abort_flag) {
  const int lane = threadIdx.x & 31;
  const bool mine = lane < kSubG && t0 + lane < nx;
  unsigned long long w[G];
  const uint64_t ts = global_ns();
  unsigned spins = 0;
  for (;;) {
    gedge_load<G>(g, t0, nx, w);
    bool ok = true;
#pragma unroll
    for (int a = 0; a < G; ++a) ok = ok && (unsigned)(w[a] >> 32) == tag;
    if (__all_sync(kFullG, !mine || ok)) return true;
    if ((++spins & 31u) == 0) {
      bool stop = false;
      if (lane == 0) stop = *abort_flag || global_ns() - ts > kWaitNsG;
      if (__shfl_sync(kFullG, stop, 0)) return false;
    }
  }
}

// Per-angle constants of a band, in registers.
template <int G> struct AngleRegs {
  float ax[G], ay[G], axy[G], gam[G], in_y[G];
};

// The 32 steps of window k of band b (stage = this window's blocks).
// first: window 0, where lanes whose column is still negative keep their
// inflow value.  Returns false if a wait gave up.  The 16 steps of a
// sub-window are unrolled (the next 16-byte group's shared-memory loads
// issue while one computes: on lognormal1024 an iteration took 11 % less
// than with 4 steps unrolled); a fully unrolled window per variant made
// the kernel's code miss the instruction caches (measured: the first
// windows of a band ran 3-10x slower than the later ones).
template <int G, bool FINAL, int PRED>
__device__ __forceinline__ bool grp_window(const GrpArgs<G> &A, const AngleRegs<G> &R, int b, int k,
                                           bool first, const float *stage, float (&psi)[G], float *edge_in,
                                           float *edge_out, int ld, volatile int *prog,
                                           volatile int *abort_flag,
                                           const unsigned long long *g_in, unsigned long long *g_out,
                                           unsigned tag, unsigned long long (&gw)[G]) {
  const int lane = threadIdx.x & 31;
  const int nx = A.nx;
  const float4 *st4 = reinterpret_cast<const float4 *>(stage + G * kBlk);
  const float4 *sp4 = reinterpret_cast<const float4 *>(stage + (G + 1) * kBlk);
  // the window's partial scalar flux replaces, float4 by float4, the
  // sigma_s phi values this lane has just read (the stage's sp block), and
  // the block is bulk-stored after the window: no generic global stores in
  // the sweep, so the progress fences wait only for shared memory
  float4 *part4 = reinterpret_cast<float4 *>(const_cast<float *>(stage) + (G + 1) * kBlk);
  // the cells this lane writes in the final sweep: row v, columns u = t - lane
  const int v = 32 * b + lane;
  const bool row_ok = v < A.ny;
  const int yrow = (A.quad & 2) ? A.ny - 1 - v : v;
#pragma unroll 1
  for (int sb = 0; sb < 32; sb += kSubG) {
    const int t0 = 32 * k + sb;
    // the lower neighbours of lane 0 for columns t0 .. t0 + kSubG - 1
    if (PRED == 2 && t0 < nx) {
      if (!gedge_take<G>(g_in, t0, nx, tag, gw, edge_in, ld, abort_flag)) return false;
    } else if (PRED == 1 && t0 < nx) {
      if (!wait_flag(prog + b - 1, min(nx, t0 + kSubG), abort_flag)) return false;
    }
#pragma unroll
    for (int qq = 0; qq < kSubG / 4; ++qq) {
      const int q = sb / 4 + qq;
      const int tq = t0 + 4 * qq;
      const int f4 = lane * 8 + (q ^ (lane & 7));
      float4 vs[G], ed[G];
#pragma unroll
      for (int a = 0; a < G; ++a) vs[a] = reinterpret_cast<const float4 *>(stage + a * kBlk)[f4];
      const float4 vt = st4[f4], vp = sp4[f4];
#pragma unroll
      for (int a = 0; a < G; ++a) {
        if (PRED) {
          // written by another warp before the wait above (whose fence and
          // warp barrier keep these loads after it)
          ed[a] = *reinterpret_cast<const float4 *>(edge_in + a * ld + tq);
        } else {
          ed[a] = make_float4(R.in_y[a], R.in_y[a], R.in_y[a], R.in_y[a]);
        }
      }
      float4 out;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int t = tq + s;
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < G; ++a) {
          const float src = f4c(vs[a], s) + f4c(vp, s);
          const float inv = rcp_approx(f4c(vt, s) + R.axy[a]);
          float down = __shfl_up_sync(kFullG, psi[a], 1);
          if (lane == 0) down = f4c(ed[a], s);
          float p = __fmul_rn(__fmaf_rn(R.ay[a], down, __fmaf_rn(R.ax[a], psi[a], src)), inv);
          if (first && t < lane) p = psi[a];
          psi[a] = p;
          acc = __fmaf_rn(R.gam[a], p, acc);
          if (lane == 31) edge_out[a * ld + t - 31] = p;
          if (FINAL) {
            const int u = t - lane;
            if (a < A.na && row_ok && u >= 0 && u < nx) {
              const int x = (A.quad & 1) ? nx - 1 - u : u;
              A.psi[a][(size_t)yrow * nx + x] = p;
            }
          }
        }
        f4s(out, s, acc);
      }
      if (!FINAL) part4[f4] = out;
    }
    if (lane == 31) {
      __threadfence_block();
      prog[b] = min(nx, max(0, t0 + kSubG - 31));
    }
    if (g_out) {
      // the unit's last band: the top-row columns finished in this
      // sub-window go to the next unit's CTA as tagged words
      __syncwarp();
      const int c = t0 - 31 + lane;
      if (lane < kSubG && (unsigned)c < (unsigned)nx) {
#pragma unroll
        for (int a = 0; a < G; ++a)
          st_relaxed_g(g_out + (size_t)c * G + a,
                       ((unsigned long long)tag << 32) | __float_as_uint(edge_out[a * ld + c]));
      }
    }
  }
  return true;
}

// One band of 32 rows of a group, swept by one warp.  pred: 0 no band below
// (the bottom inflow), 1 the band below is in this CTA, 2 in another CTA.
template <int G, bool FINAL, int PRED>
__device__ __forceinline__ bool grp_band(const GrpArgs<G> &Ain, int b, const GrpSmem &S, Pipe &P,
                                         const unsigned long long *g_in, unsigned long long *g_out,
                                         unsigned tag, volatile int *abort_flag) {
  const GrpArgs<G> &A = Ain;
  AngleRegs<G> R;
#pragma unroll
  for (int a = 0; a < G; ++a) {
    R.ax[a] = A.ax[a];
    R.ay[a] = A.ay[a];
    R.axy[a] = A.axy[a];
    R.gam[a] = A.gam[a];
    R.in_y[a] = A.in_y[a];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int NS = S.S;
  float *stages = S.stages + (size_t)wid * NS * (G + 2) * kBlk;
  uint64_t *mb = S.mbar + wid * NS;
  const int ld = S.edge_ld;
  float *edge_out = S.edge + (size_t)(b % (kNWg + 1)) * G * ld + kEdgePadG;
  float *edge_in = S.edge + (size_t)((b + kNWg) % (kNWg + 1)) * G * ld + kEdgePadG;
  volatile int *prog = S.prog;
  const int nwin = A.nwin;
  float psi[G];
#pragma unroll
  for (int a = 0; a < G; ++a) psi[a] = A.in_x[a];
  unsigned long long gw[G];
#pragma unroll
  for (int a = 0; a < G; ++a) gw[a] = 0ull;
  if (PRED == 2) {
    // start two sub-windows later than the band below allows: the words a
    // sub-window needs were then written well before they are loaded, and
    // the loads rarely have to be repeated
    if (2 * kSubG < A.nx && !gedge_ready<G>(g_in, 2 * kSubG, A.nx, tag, abort_flag)) {
      __syncwarp();
      return false;
    }
    gedge_load<G>(g_in, 0, A.nx, gw);
  }
  // windows 0 .. NS-2 into their stages (after the previous band's bulk
  // stores have read them)
  __syncwarp();
  fence_proxy_async();
  if (lane == 0) {
    bulk_wait_read();
    for (int k = 0; k < NS - 1 && k < nwin; ++k) issue_window<G>(A, b, k, stages + (size_t)k * (G + 2) * kBlk, mb + k);
  }
  int issued = min(NS - 1, nwin);  // windows issued so far
  bool ok = true;
  int k = 0;
  for (; k < nwin; ++k) {
    // the stage of window k - 1 is free again: window k + NS - 1 goes there
    if (k + NS - 1 < nwin) {
      __syncwarp();
      fence_proxy_async();
      const int sn = (k + NS - 1) % NS;
      if (lane == 0) {
        bulk_wait_read();  // the partial stored from this stage has left it
        issue_window<G>(A, b, k + NS - 1, stages + (size_t)sn * (G + 2) * kBlk, mb + sn);
      }
      ++issued;
    }
    const int sc = k % NS;
    if (!wait_stage(mb + sc, (P.parity >> sc) & 1u, abort_flag)) { ok = false; break; }
    P.parity ^= 1u << sc;
    const float *stage = stages + (size_t)sc * (G + 2) * kBlk;
    const bool w_ok = grp_window<G, FINAL, PRED>(A, R, b, k, k == 0, stage, psi, edge_in, edge_out, ld,
                                                  prog, abort_flag, g_in, g_out, tag, gw);
    if (!w_ok) { ok = false; ++k; break; }
    if (!FINAL) {
      __syncwarp();
      fence_proxy_async();
      if (lane == 0)
        bulk_store(A.part + ((size_t)b * nwin + k) * kBlk, stage + (G + 1) * kBlk, kBlk * 4, policy_evict_last());
    }
  }
  // the partials are in global memory before the scalar-flux phase reads
  // them (after the grid barrier)
  if (lane == 0) {
    bulk_wait_all();
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  if (!ok) {
    // copies still in flight into this warp's stages must land before the
    // stages are reused or the CTA exits: windows k .. issued - 1 (the
    // window whose wait gave up included)
    for (int kk = k; kk < issued; ++kk) {
      const int sc = kk % NS;
      drain_stage(mb + sc, (P.parity >> sc) & 1u);
      P.parity ^= 1u << sc;
    }
  }
  __syncwarp();
  return ok;
}

// The group's arguments for instance I (sigma_s phi / 4 pi of parity par).
__device__ GrpArgs<kGA> grp_args(const Inst &I, int g, int par, bool final_sweep) {
  GrpArgs<kGA> A;
  const int *rec = I.grp_tab + g * kGrpRec;
  A.nx = I.nx;
  A.ny = I.ny;
  A.nwin = I.nwin;
  A.quad = rec[0];
  A.na = rec[1];
  const double *gam = I.gamma_ext ? I.gamma_ext : I.small + I.lay.gamma;
  for (int a = 0; a < kGA; ++a) {
    // a group with fewer angles repeats its first angle's direction with
    // weight 0 (its unused source slot holds finite values: zero at first)
    const int j = rec[2 + (a < A.na ? a : 0)];
    const int kq = I.idx[j];
    const double ox = I.ox[kq], oy = I.oy[kq];
    A.ax[a] = float(fabs(ox) / I.hx);
    A.ay[a] = float(fabs(oy) / I.hy);
    A.axy[a] = A.ax[a] + A.ay[a];
    A.gam[a] = a < A.na ? float(gam[j]) : 0.f;
    A.in_x[a] = float(ox > 0 ? I.psi_edge[0] : (ox < 0 ? I.psi_edge[1] : 0.0));
    A.in_y[a] = float(oy > 0 ? I.psi_edge[2] : (oy < 0 ? I.psi_edge[3] : 0.0));
    A.psi[a] = final_sweep ? as<float>(I.Psi) + (size_t)I.N * j : nullptr;
  }
  A.sg = I.sgk + grp_sgk(I.glay, g, 0, 0);
  A.sp = I.spk + ((size_t)par * 4 + A.quad) * I.glay;
  A.part = final_sweep ? nullptr : I.part + (size_t)g * I.glay;
  return A;
}

// Bands b0 .. b0 + nb - 1 of group g by one CTA (warp w: bands b0 + w,
// b0 + w + NW, ...).  Returns, in every thread of the CTA, false if a wait
// of any warp gave up.
template <bool FINAL>
__device__ bool grp_unit(const Inst &I, const SiUnit &U, int par, const GrpSmem &S, Pipe &P,
                         const unsigned long long *g_in, unsigned long long *g_out, unsigned tag,
                         volatile int *abort_flag) {
  __syncthreads();
  for (int i = U.b0 + threadIdx.x; i < U.b0 + U.nb; i += blockDim.x) S.prog[i] = 0;
  __syncthreads();
  bool ok = true;
  if (I.grp_tab[U.angle * kGrpRec + 1] > 0) {
    const GrpArgs<kGA> A = grp_args(I, U.angle, par, FINAL);
    const int wid = threadIdx.x >> 5;
    for (int b = U.b0 + wid; wid < kNWg && b < U.b0 + U.nb && ok; b += kNWg) {
      const int pred = b == 0 ? 0 : (b == U.b0 ? (g_in ? 2 : 0) : 1);
      unsigned long long *go = b == U.b0 + U.nb - 1 ? g_out : nullptr;
      if (pred == 1) ok = grp_band<kGA, FINAL, 1>(A, b, S, P, nullptr, go, tag, abort_flag);
      else if (pred == 2) ok = grp_band<kGA, FINAL, 2>(A, b, S, P, g_in, go, tag, abort_flag);
      else ok = grp_band<kGA, FINAL, 0>(A, b, S, P, nullptr, go, tag, abort_flag);
    }
  }
  if (!ok) *abort_flag = 1;
  return __syncthreads_and(ok) != 0;
}

// Phase A of one iteration (or the final sweep): every unit of the active
// instances.  Returns false when a wait gave up.
template <bool FINAL>
__device__ bool grp_sweeps(const Inst *__restrict__ insts, const SiCtl &ctl, int n_units, const int *active,
                           const int *par_of, unsigned ctr, unsigned tag, const GrpSmem &S, Pipe &P,
                           volatile int *abort_flag) {
  __shared__ int unit_g;
  for (;;) {
    if (threadIdx.x == 0) unit_g = (int)atomicAdd(ctl.work + ctr, 1u);
    __syncthreads();
    const int u = unit_g;
    __syncthreads();
    if (u >= n_units) return true;
    const SiUnit U = ctl.units[u];
    if (!active[U.inst]) continue;
    const unsigned long long *g_in = U.in_row >= 0 ? ctl.gedge + (size_t)U.in_row * ctl.gedge_ld : nullptr;
    unsigned long long *g_out = U.out_row >= 0 ? ctl.gedge + (size_t)U.out_row * ctl.gedge_ld : nullptr;
    if (!grp_unit<FINAL>(insts[U.inst], U, par_of[U.inst], S, P, g_in, g_out, tag, abort_flag)) return false;
  }
}

}  // namespace

// ------------------------------------------------------------------
// The source iteration as a loop of kernels (a while node of the step's
// CUDA graph): k_grp_sweep (the sweeps of all active groups), k_grp_qsum
// (per quadrant, the sum of its groups' partials), k_grp_phi (phi, the next
// sigma_s phi / 4 pi, the convergence test; its last block decides per
// instance and ends the loop); after the loop k_grp_sweep<true> writes Psi
// from each instance's last sigma_s phi.  The sweep needs no co-resident
// grid: a unit is claimed only by a running CTA, after the unit it waits
// on.  The scalar-flux kernels run at full occupancy.
// ------------------------------------------------------------------

// Resets the loop state before a step's source iteration.
__global__ void k_grp_prep(const Inst *__restrict__ insts, int n, SiCtl ctl, GrpSi *gs) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    ctl.work[0] = 0u;
    ctl.work[1] = 0u;
    *ctl.abort_flag = 0;
    *ctl.epoch += 1u;  // stale edge words of earlier launches never match
    gs->it = 0;
    gs->done = 0u;
  }
  if (t < n) {
    insts[t].conv[0] = 0ull;
    insts[t].conv[1] = 0ull;
    *insts[t].nonpos = 0;
    gs->active[t] = *insts[t].status == kOk ? 1 : 0;
    gs->par_of[t] = -1;
    relax_reset(gs->relax + 3 * t);
  }
}

template <bool FINAL>
__global__ void __launch_bounds__(kNWg * 32)
k_grp_sweep(const Inst *__restrict__ insts, SiCtl ctl, GrpSi *gs, int stages) {
  extern __shared__ __align__(128) unsigned char smem[];
  GrpSmem S;
  S.S = stages;
  size_t off = 0;
  S.stages = reinterpret_cast<float *>(smem + off);
  off += (size_t)kNWg * stages * (kGA + 2) * kBlk * 4;
  S.mbar = reinterpret_cast<uint64_t *>(smem + off);
  off += ((size_t)kNWg * stages * 8 + 15) / 16 * 16;
  S.edge_ld = edge_ld_g(ctl.nx_max);
  S.edge = reinterpret_cast<float *>(smem + off);
  off += (size_t)(kNWg + 1) * kGA * S.edge_ld * 4;
  S.prog = reinterpret_cast<int *>(smem + off);
  off += (size_t)(ctl.bands_max + 3) / 4 * 4 * 4;
  int *act = reinterpret_cast<int *>(smem + off);
  off += (size_t)(ctl.n_inst + 3) / 4 * 4 * 4;
  int *par = reinterpret_cast<int *>(smem + off);
  volatile int *abort_flag = ctl.abort_flag;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int s = 0; s < stages; ++s) mbar_init(S.mbar + wid * stages + s, 1);
  for (int i = threadIdx.x; i < (kNWg + 1) * kGA * S.edge_ld; i += blockDim.x) S.edge[i] = 0.f;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const int it = *(volatile int *)&gs->it;
  for (int i = threadIdx.x; i < ctl.n_inst; i += blockDim.x) {
    if (FINAL) {
      // instances swept in this step's iteration, unless a wait gave up
      const int st = *insts[i].status;
      act[i] = gs->par_of[i] >= 0 && (st == kOk || st == kENotConv);
      par[i] = gs->par_of[i];
    } else {
      act[i] = gs->active[i];
      par[i] = it & 1;
    }
  }
  __syncthreads();
  if (*abort_flag) return;
  Pipe P;
  P.parity = 0u;
  const unsigned tag = ((*(volatile unsigned *)ctl.epoch & 0xfffffu) << 12) |
                       ((unsigned)(it + (FINAL ? 2 : 1)) & 0xfffu);
  grp_sweeps<FINAL>(insts, ctl, gs->n_units, act, par, it & 1, tag, S, P, abort_flag);
}

// Per quadrant of each active instance, the sum of its groups' partials
// (the groups are ordered by quadrant; each sum in group order), 16 bytes
// at a time.
__global__ void __launch_bounds__(256) k_grp_qsum(const Inst *__restrict__ insts, int n, const GrpSi *gs) {
  for (int i = 0; i < n; ++i) {
    if (!gs->active[i]) continue;
    const Inst &I = insts[i];
    const size_t n4 = I.glay / 4;
    int lo = 0;
    for (int q = 0; q < 4; ++q) {
      int hi = lo;
      while (hi < I.grp_ng && I.grp_tab[hi * kGrpRec + 1] > 0 && I.grp_tab[hi * kGrpRec] == q) ++hi;
      if (hi > lo) {
        const float4 *src = reinterpret_cast<const float4 *>(I.part);
        float4 *dst = reinterpret_cast<float4 *>(I.qsum + (size_t)q * I.glay);
        for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4;
             e += (size_t)gridDim.x * blockDim.x) {
          float4 acc = src[(size_t)lo * n4 + e];
          for (int g = lo + 1; g < hi; ++g) {
            const float4 v = src[(size_t)g * n4 + e];
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
          }
          dst[e] = acc;
        }
      }
      lo = hi;
    }
  }
}

// phi = the quadrant sums at each cell, sigma_s phi / 4 pi of the next
// iteration in the four quadrant layouts, the convergence maxima; the last
// block to finish takes every instance's decision (as the per-angle
// kernel's), resets the counters of the next iteration and, when no
// instance is left (or a wait gave up), ends the loop.
__global__ void __launch_bounds__(256) k_grp_phi(const Inst *__restrict__ insts, int n, SiCtl ctl, GrpSi *gs,
                                                 cudaGraphConditionalHandle loop) {
  const int it = gs->it;
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < n; ++i) {
    if (!gs->active[i]) continue;
    const Inst &I = insts[i];
    const int nx = I.nx, ny = I.ny, N = I.N, nwin = I.nwin;
    int qmask = 0;  // quadrants with a group
    for (int g = 0; g < I.grp_ng; ++g)
      if (I.grp_tab[g * kGrpRec + 1] > 0) qmask |= 1 << I.grp_tab[g * kGrpRec];
    const float *qs = I.qsum;
    const float *ss4 = as_c<float>(I.ss4);
    const float *pold = as_c<float>((it & 1) ? I.phi1 : I.phi0);
    float *pnew = as<float>((it & 1) ? I.phi0 : I.phi1);
    float *spn = I.spk + (size_t)((it + 1) & 1) * 4 * I.glay;
    const float om = (float)gs->relax[3 * i];  // relaxation (1: the plain iteration)
    float dmax = 0.f, pmax = 0.f;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
      const int y = c / nx, x = c - y * nx;
      unsigned o[4];
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        o[q] = (unsigned)grp_off(q, nx, ny, nwin, x, y);
        v[q] = (qmask >> q) & 1 ? qs[(size_t)q * I.glay + o[q]] : 0.f;
      }
      const float acc = ((v[0] + v[1]) + v[2]) + v[3];
      const float po = pold[c];
      const float pn = om == 1.f ? acc : fmaf(om, acc - po, po);
      pnew[c] = pn;
      const float sp = ss4[c] * pn;
#pragma unroll
      for (int q = 0; q < 4; ++q) spn[(size_t)q * I.glay + o[q]] = sp;
      dmax = fmaxf(dmax, fabsf(acc - po));
      pmax = fmaxf(pmax, fabsf(acc));
      if (!isfinite(acc)) dmax = INFINITY;  // diverged (fmaxf drops NaN)
    }
    dmax = warp_max(dmax);
    pmax = warp_max(pmax);
    if (lane == 0) {
      atomic_max_nonneg(I.conv + (it & 1) * 2 + 0, (double)dmax);
      atomic_max_nonneg(I.conv + (it & 1) * 2 + 1, (double)pmax);
    }
  }
  // the last block to finish decides
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&gs->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  const bool aborted = *(volatile int *)ctl.abort_flag != 0;
  int left = 0;
  for (int i = 0; i < n; ++i) {
    if (!gs->active[i]) continue;
    const Inst &I = insts[i];
    gs->par_of[i] = it & 1;  // the parity of this instance's last sweep so far
    if (aborted) {
      set_status(I.status, kETimeout);
      gs->active[i] = 0;
      continue;
    }
    volatile unsigned long long *cv = I.conv + (it & 1) * 2;
    const double d = __longlong_as_double((long long)cv[0]);
    const double m = __longlong_as_double((long long)cv[1]);
    const int done_iters = it + 1;
    bool done;
    if (gs->force_iters > 0) {
      done = done_iters >= gs->force_iters;
      if (done) gs->active[i] = 0;
      else ++left;
      I.conv[((it + 1) & 1) * 2 + 0] = 0ull;
      I.conv[((it + 1) & 1) * 2 + 1] = 0ull;
      continue;
    }
    const bool diverged = relax_track(d, m, gs->relax + 3 * i);  // true: diverging even when relaxed
    if (diverged || !(d <= 1.0e308)) {  // or a non-finite scalar flux
      done = true;
      set_status(I.status, kENotConv);
    } else if (I.fixed_iters > 0) {
      done = done_iters >= I.fixed_iters;
    } else {
      done = d <= I.si_tol * m;
      if (!done && done_iters >= I.max_iter) {
        done = true;
        set_status(I.status, kENotConv);
      }
    }
    if (done) {
      gs->active[i] = 0;
      *I.iters = done_iters;
      atomicAdd(I.iters_total, (unsigned long long)done_iters);
    } else {
      ++left;
    }
    I.conv[((it + 1) & 1) * 2 + 0] = 0ull;
    I.conv[((it + 1) & 1) * 2 + 1] = 0ull;
  }
  ctl.work[(it + 1) & 1] = 0u;
  gs->done = 0u;
  gs->it = it + 1;
  __threadfence();
  if (left == 0) cudaGraphSetConditional(loop, 0);
}

// ------------------------------------------------------------------
// host-side launch helpers
// ------------------------------------------------------------------
size_t si_grp_smem_bytes(int nx_max, int bands_max, int n_inst, int stages) {
  return (size_t)kNWg * stages * (kGA + 2) * kBlk * 4 + ((size_t)kNWg * stages * 8 + 15) / 16 * 16 +
         (size_t)(kNWg + 1) * kGA * edge_ld_g(nx_max) * 4 + (size_t)(bands_max + 3) / 4 * 4 * 4 +
         2 * (size_t)(n_inst + 3) / 4 * 4 * 4;
}

// The stage count (3, else 2) that fits the device's shared memory per
// block, or 0 if not even 2 fit.
int si_grp_stages(int nx_max, int bands_max, int n_inst) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int s = 3; s >= 2; --s)
    if (si_grp_smem_bytes(nx_max, bands_max, n_inst, s) <= (size_t)optin) return s;
  return 0;
}

// CTAs of the sweep kernel: as many as fit at once (they claim units).
int si_grp_max_grid(int nx_max, int bands_max, int n_inst, int stages) {
  const size_t smem = si_grp_smem_bytes(nx_max, bands_max, n_inst, stages);
  for (auto fn : {k_grp_sweep<false>, k_grp_sweep<true>})
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grp_sweep<false>, kNWg * 32, smem) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

cudaError_t launch_grp_prep(const Inst *d, int n, const SiCtl &ctl, GrpSi *gs, cudaStream_t st) {
  return launch_pdl(k_grp_prep, dim3((n + 255) / 256), dim3(256), 0, st, d, n, ctl, gs);
}

// The body of the loop (three kernels) on stream st: used to fill the while
// node's body graph by stream capture.
cudaError_t launch_grp_iteration(const Inst *d, int n, const SiCtl &ctl, GrpSi *gs, int grid, int stages,
                                 cudaGraphConditionalHandle loop, cudaStream_t st) {
  const size_t smem = si_grp_smem_bytes(ctl.nx_max, ctl.bands_max, ctl.n_inst, stages);
  k_grp_sweep<false><<<grid, kNWg * 32, smem, st>>>(d, ctl, gs, stages);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_grp_qsum<<<4 * sms, 256, 0, st>>>(d, n, gs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_grp_phi<<<4 * sms, 256, 0, st>>>(d, n, ctl, gs, loop);
  return cudaGetLastError();
}

cudaError_t launch_grp_final(const Inst *d, const SiCtl &ctl, GrpSi *gs, int grid, int stages, cudaStream_t st) {
  const size_t smem = si_grp_smem_bytes(ctl.nx_max, ctl.bands_max, ctl.n_inst, stages);
  k_grp_sweep<true><<<grid, kNWg * 32, smem, st>>>(d, ctl, gs, stages);
  return cudaGetLastError();
}

int si_grp_warps() { return kNWg; }
int si_grp_lag() { return 32 + kSubG; }

}  // namespace dlr
