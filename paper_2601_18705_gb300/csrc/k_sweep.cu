// k_sweep.cu -- the hot path of Algorithm 1 step 4: DG0 upwind transport
// sweeps at the r collocation angles with source iteration on
//   Om^(j).grad psi_j + (sigma + 1/(c dt)) psi_j
//       = sigma_s/(4 pi) beta^T What^{-1} Psi + q + psi0_j / (c dt)
// (Eq. steady state collocation of Haut et al.; phi = beta^T What^{-1} Psi is
// evaluated as gamma^T Psi with gamma = What^{-T} beta).
//
// Sweep organisation (one CTA per (instance, angle) unit):
//   * cells are visited in sweep coordinates (u, v): x and y are mirrored so
//     that the direction points to +u, +v;
//   * rows are grouped in bands of 32; lane i of a warp owns row 32b+i and at
//     step t updates column u = t - i (an anti-diagonal wavefront); the value
//     of the cell below arrives from lane i-1 by a warp shuffle, the value of
//     the cell to the left stays in a register;
//   * the inputs of each 32 x 32 chunk (lane = column) are prefetched into
//     registers one chunk ahead and staged as (source, 1/(sigma_t + ax +
//     ay)) in a per-warp ring of 64 diagonal slots: cell (row i, column u)
//     goes to slot (u + i) mod 64, so at step t every lane reads slot
//     t mod 64 (a compile-time offset inside an unrolled window of 32
//     steps) and writes its result back there; rows of a slot are padded to
//     33 entries, which keeps staging and stepping free of bank conflicts;
//     a chunk's results are written out when its slots are reused;
//   * only the first window and the last ones need per-lane masks; the
//     others run a mask-free step of two loads, one shuffle, three FP
//     operations and two stores;
//   * the top row of a band is handed to the next band (another warp) through
//     a shared-memory ring of row buffers, guarded by a per-band progress
//     counter published every kSub steps; every wait is bounded in time.
// The source-iteration loop runs inside one cooperative launch per step for
// all instances: sweep phase, grid barrier, scalar-flux phase
// phi = sum_j gamma_j psi_j with the convergence test, grid barrier.
#include "dlr_internal.cuh"
#include "k_dsa.cuh"

namespace dlr {

// NW: sweeping warps per CTA.  kSub: progress granularity (steps).  Finer
// steps shorten the lag between bands (31 + kSub steps) but their waits, edge
// reads and progress stores cost more than the lag saves: in FP32 a whole
// window (measured: 8 -> 32 cut lognormal1024 from 23.2 to 16.4 ms per
// step).  In FP64 the kSub staged (source, 1/diagonal) pairs held across a
// sub-window cost 4 registers each: at 16 or 32 the kernel spills kilobytes
// (measured at 32: checker256 FP64 5.2 -> 5.8 ms per step), so it keeps 8.
template <typename real> struct SweepCfg;
template <> struct SweepCfg<float> { static constexpr int NW = 8, kSub = 32; };
template <> struct SweepCfg<double> { static constexpr int NW = 4, kSub = 8; };
constexpr uint64_t kWaitNs = 4000000000ull;    // bound of any single wait
constexpr unsigned kFull = 0xffffffffu;

template <typename real>
struct SweepArgs {
  int nx, ny;
  bool flipx, flipy;
  real ax, ay, in_x, in_y;
  const real *sig_t;  // N
  const real *src;    // N: the angle's fixed source
  const real *sphi;   // N or nullptr: sigma_s phi / (4 pi), added to src
  real *psi;          // N: output
};

constexpr int kRing = 64;    // diagonal slots per warp
constexpr int kRingLd = 33;  // entries per slot (32 lanes, padded)

// Edge rows (a band's top row for the next band) hold column u at index
// u + kEdgePad; the padding absorbs the writes of columns -31..-1 and
// nx..nx+31 that the mask-free steps produce, and the vector reads of
// kSub columns past nx.
constexpr int kEdgePad = 32;
__host__ __device__ inline int edge_ld(int nx_max) { return (nx_max + 3) / 4 * 4 + 2 * kEdgePad; }

template <typename real> struct Real4;
template <> struct Real4<float> {
  using type = float4;
  static constexpr int kN = 4;
  __device__ static void unpack(const volatile float4 &v, float *o) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <> struct Real4<double> {
  using type = double2;
  static constexpr int kN = 2;
  __device__ static void unpack(const volatile double2 &v, double *o) {
    o[0] = v.x; o[1] = v.y;
  }
};

struct SweepSmem {
  void *tiles;    // NW warps x kRing x kRingLd real2
  void *edge;     // (NW + 1) x edge_ld(nx_max) real
  int *prog;      // bands_max
  int edge_ld;
};

// Bounded wait of lane 0 until *flag >= need.  The polls back off with
// __nanosleep, so a waiting warp takes (almost) no issue slots from the
// warps that are sweeping on the same scheduler.  Returns false on timeout
// or abort (the warp then leaves the unit).
__device__ __forceinline__ bool wait_progress(volatile int *flag, int need,
                                              volatile int *abort_flag) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) {
    if (*flag < need) {
      uint64_t t0 = global_ns();
      unsigned spins = 0, nap = 16;
      while (*flag < need) {
        __nanosleep(nap);
        nap = min(nap * 2, 128u);
        if ((++spins & 63u) == 0) {
          if (*abort_flag || global_ns() - t0 > kWaitNs) { ok = false; break; }
        }
      }
    }
    __threadfence_block();
  }
  ok = __shfl_sync(kFull, ok, 0);
  __syncwarp();
  return ok;
}

// Raw inputs of one 32 x 32 chunk of a band, prefetched into registers
// (lane = column) one chunk ahead of the wavefront.  The loads use clamped,
// always valid addresses and nothing consumes their values until the chunk
// is staged, so their latency overlaps the sweep of the previous chunk.  In
// FP32 the scalar-flux source is kept apart (added when staging); in FP64 it
// is added at once to stay within the register budget.
template <typename real> struct ChunkRegs;
template <> struct ChunkRegs<float> {
  static constexpr bool kRaw = true;
  float src[32], sp[32], st[32];
};
template <> struct ChunkRegs<double> {
  static constexpr bool kRaw = false;
  double src[32], st[32];
  double sp[1];
};

// 1 / x: IEEE division in FP64; in FP32 the approximate reciprocal of the
// special-function unit (one instruction, relative error about 2^-23),
// inside the mixed-precision error budget (x = sigma_t + ax + ay >= 1 is
// never subnormal).
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Cell of the band's first row in sweep column u (index iy * nx + ix); the
// band's rows follow at multiples of row_step = +-nx.
template <typename real>
__device__ __forceinline__ int chunk_cell0(const SweepArgs<real> &A, int b, int u) {
  const int ix = A.flipx ? A.nx - 1 - u : u;
  return (A.flipy ? (A.ny - 1 - 32 * b) * A.nx : 32 * b * A.nx) + ix;
}

// FULL: the chunk is whole (32 rows and 32 columns inside the mesh), so no
// clamps or masks are needed; SP: a scalar-flux source is present.
template <typename real, bool FULL, bool SP>
__device__ __forceinline__ void load_chunk_t(const SweepArgs<real> &A, int b, int k, ChunkRegs<real> &R) {
  const int lane = threadIdx.x & 31;
  const int c0 = chunk_cell0(A, b, FULL ? 32 * k + lane : min(32 * k + lane, A.nx - 1));
  const int rs = A.flipy ? -A.nx : A.nx;
  const int last = FULL ? 31 : min(32, A.ny - 32 * b) - 1;
  const real *__restrict__ ps = A.src + c0;
  const real *__restrict__ pt = A.sig_t + c0;
  const real *__restrict__ pp = SP ? A.sphi + c0 : nullptr;
#pragma unroll
  for (int ii = 0; ii < 32; ++ii) {
    const int off = (FULL ? ii : min(ii, last)) * rs;
    R.src[ii] = ps[off];
    R.st[ii] = pt[off];
    if (SP) {
      if (ChunkRegs<real>::kRaw) R.sp[ChunkRegs<real>::kRaw ? ii : 0] = pp[off];
      else R.src[ii] += pp[off];
    }
  }
}

template <typename real>
__device__ __forceinline__ bool chunk_full(const SweepArgs<real> &A, int b, int k) {
  return 32 * b + 32 <= A.ny && 32 * k + 32 <= A.nx;
}

template <typename real>
__device__ __forceinline__ void load_chunk(const SweepArgs<real> &A, int b, int k, ChunkRegs<real> &R) {
  const bool full = chunk_full(A, b, k);
  if (A.sphi) {
    if (full) load_chunk_t<real, true, true>(A, b, k, R);
    else load_chunk_t<real, false, true>(A, b, k, R);
  } else {
    if (full) load_chunk_t<real, true, false>(A, b, k, R);
    else load_chunk_t<real, false, false>(A, b, k, R);
  }
}

// Ring entry of (row ii, column u = 32k + lane): slot (u + ii) mod 64, entry
// ii, i.e. ring + (32 PAR + lane) * 33 + 34 ii for PAR = k mod 2, minus one
// ring length once 32 PAR + lane + ii reaches 64 (odd chunks only).
template <int PAR>
__device__ __forceinline__ int ring_entry(int lane, int ii) {
  int e = (32 * PAR + lane) * kRingLd + (kRingLd + 1) * ii;
  if (PAR == 1 && ii >= 32 - lane) e -= kRing * kRingLd;
  return e;
}

// (source, 1 / (sigma_t + ax + ay)) of a prefetched chunk into its diagonal
// slots.  Cells outside the mesh get a zero source and sigma_t = 1.
template <typename real, bool FULL, bool SP, int PAR>
__device__ __forceinline__ void stage_chunk_t(const SweepArgs<real> &A, const ChunkRegs<real> &R, int b,
                                              int k, typename Real2<real>::type *ring) {
  const int lane = threadIdx.x & 31;
  const real axy = A.ax + A.ay;
  const bool col_ok = FULL || 32 * k + lane < A.nx;
  const int rows = FULL ? 32 : min(32, A.ny - 32 * b);
#pragma unroll
  for (int ii = 0; ii < 32; ++ii) {
    const bool ok = FULL || (col_ok && ii < rows);
    real src = R.src[ii];
    if (SP && ChunkRegs<real>::kRaw) src += R.sp[ChunkRegs<real>::kRaw ? ii : 0];
    typename Real2<real>::type e;
    e.x = ok ? src : real(0);
    e.y = recip((ok ? R.st[ii] : real(1)) + axy);
    ring[ring_entry<PAR>(lane, ii)] = e;
  }
}

template <typename real>
__device__ __forceinline__ void stage_chunk(const SweepArgs<real> &A, const ChunkRegs<real> &R, int b,
                                            int k, typename Real2<real>::type *ring) {
  const bool full = chunk_full(A, b, k), sp = A.sphi != nullptr;
#define DLR_STAGE(F, S)                                                 \
  do {                                                                  \
    if (k & 1) stage_chunk_t<real, F, S, 1>(A, R, b, k, ring);          \
    else stage_chunk_t<real, F, S, 0>(A, R, b, k, ring);                \
  } while (0)
  if (full) {
    if (sp) DLR_STAGE(true, true); else DLR_STAGE(true, false);
  } else {
    if (sp) DLR_STAGE(false, true); else DLR_STAGE(false, false);
  }
#undef DLR_STAGE
}

// results of chunk k (complete) from their diagonal slots to psi
template <typename real, bool FULL, int PAR>
__device__ __forceinline__ void write_chunk_t(const SweepArgs<real> &A, int b, int k,
                                              const typename Real2<real>::type *ring) {
  const int lane = threadIdx.x & 31;
  const int u = 32 * k + lane;
  if (!FULL && u >= A.nx) return;
  real *__restrict__ out = A.psi + chunk_cell0(A, b, u);
  const int rs = A.flipy ? -A.nx : A.nx;
  const int rows = FULL ? 32 : min(32, A.ny - 32 * b);
#pragma unroll
  for (int ii = 0; ii < 32; ++ii)
    if (FULL || ii < rows) out[ii * rs] = ring[ring_entry<PAR>(lane, ii)].x;
}

template <typename real>
__device__ __forceinline__ void write_chunk(const SweepArgs<real> &A, int b, int k,
                                            const typename Real2<real>::type *ring) {
  if (chunk_full(A, b, k)) {
    if (k & 1) write_chunk_t<real, true, 1>(A, b, k, ring);
    else write_chunk_t<real, true, 0>(A, b, k, ring);
  } else {
    if (k & 1) write_chunk_t<real, false, 1>(A, b, k, ring);
    else write_chunk_t<real, false, 0>(A, b, k, ring);
  }
}

// Edge rows between units of one angle (an angle whose bands are split over
// several CTAs) live in global memory as tagged words: column c of the row
// is one (FP32) or two (FP64) 64-bit words tag << 32 | 32 bits of the value,
// each written and read as a single relaxed access, so a reader that sees
// the expected tag (launch epoch, iteration) also sees the value, with no
// fence or flag on either side.  The producer is the unit's last band, which
// copies the kSub top-row values of each sub-window from its shared edge row
// (kSub lanes, one store each, outside the step loop); the consumer is the
// unit's first band, which loads the words of the next kSub columns one
// sub-window ahead and checks their tags.
struct EdgeLink {
  int b0, nb;                        // the unit's bands
  const unsigned long long *g_in;    // words of band b0 - 1's top row (nullptr: none)
  unsigned long long *g_out;         // words of band b0 + nb - 1's top row (nullptr: none)
  unsigned tag;
};

template <typename real> struct EdgeWords;
template <> struct EdgeWords<float> {
  static constexpr int kW = 1;
  __device__ static float decode(const unsigned long long *w) { return __uint_as_float((unsigned)w[0]); }
  __device__ static void encode(float v, unsigned long long tag, unsigned long long *w) {
    w[0] = tag | __float_as_uint(v);
  }
};
template <> struct EdgeWords<double> {
  static constexpr int kW = 2;
  __device__ static double decode(const unsigned long long *w) {
    return __hiloint2double((int)(unsigned)w[1], (int)(unsigned)w[0]);
  }
  __device__ static void encode(double v, unsigned long long tag, unsigned long long *w) {
    w[0] = tag | (unsigned)__double2loint(v);
    w[1] = tag | (unsigned)__double2hiint(v);
  }
};

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v));
}

template <typename real>
__device__ __forceinline__ void edge_load(const unsigned long long *g, int t0, int nx,
                                          unsigned long long (&w)[EdgeWords<real>::kW]) {
  constexpr int kSub = SweepCfg<real>::kSub;
  const int lane = threadIdx.x & 31, c = t0 + lane;
  if (lane < kSub && c < nx) {
#pragma unroll
    for (int q = 0; q < EdgeWords<real>::kW; ++q) w[q] = ld_relaxed(g + (size_t)c * EdgeWords<real>::kW + q);
  }
}

// Lane 0's lower neighbours for columns t0 .. t0 + kSub - 1 from the tagged
// words prefetched in w (reloaded until every tag matches, bounded in time),
// then the prefetch of the next sub-window.
template <typename real>
__device__ __forceinline__ bool edge_take(const unsigned long long *g, int t0, int nx, unsigned tag,
                                          unsigned long long (&w)[EdgeWords<real>::kW],
                                          real (&ed)[SweepCfg<real>::kSub], volatile int *abort_flag) {
  constexpr int kW = EdgeWords<real>::kW, kSub = SweepCfg<real>::kSub;
  const int lane = threadIdx.x & 31;
  const bool mine = lane < kSub && t0 + lane < nx;
  auto valid = [&]() {
    bool ok = true;
#pragma unroll
    for (int q = 0; q < kW; ++q) ok = ok && (unsigned)(w[q] >> 32) == tag;
    return !mine || ok;
  };
  if (!__all_sync(kFull, valid())) {
    const uint64_t ts = global_ns();
    unsigned nap = 32, spins = 0;
    do {
      __nanosleep(nap);
      nap = min(nap * 2, 256u);
      edge_load<real>(g, t0, nx, w);
      if ((++spins & 15u) == 0) {
        bool stop = false;
        if (lane == 0) stop = *abort_flag || global_ns() - ts > kWaitNs;
        if (__shfl_sync(kFull, stop, 0)) return false;
      }
    } while (!__all_sync(kFull, valid()));
  }
  const real v = EdgeWords<real>::decode(w);
#pragma unroll
  for (int s = 0; s < kSub; ++s) ed[s] = __shfl_sync(kFull, v, s);
  edge_load<real>(g, t0 + kSub, nx, w);
  return true;
}

// The 32 steps t = 32k + tau of window k (OFF = 32 (k mod 2): slot t mod 64
// = OFF + tau).  Lane i updates column u = t - i.  FIRST (window 0): lanes
// whose column is still negative keep their inflow value; in later windows
// every column is >= 0, and columns >= nx only touch slots and edge entries
// that nobody reads, so no lane needs a mask.
template <typename real, int NW, int OFF, bool FIRST, bool GIN>
__device__ __forceinline__ bool sweep_window(int b, int k, const SweepArgs<real> &A,
                                             typename Real2<real>::type *mine, real &psi,
                                             const real *edge_in, real *edge_out,
                                             volatile int *prog, volatile int *abort_flag,
                                             const unsigned long long *g_in,
                                             unsigned long long *g_out, unsigned tag,
                                             unsigned long long (&gw)[EdgeWords<real>::kW]) {
  constexpr int kSub = SweepCfg<real>::kSub;
  const int lane = threadIdx.x & 31;
  const int nx = A.nx;
  const real ax = A.ax, ay = A.ay;
#pragma unroll
  for (int sb = 0; sb < 32; sb += kSub) {
    const int t0 = 32 * k + sb;
    // the sub-window's staged (source, 1 / diagonal) entries, loaded before
    // the wait: the steps below only overwrite entries already read
    typename Real2<real>::type vv[kSub];
#pragma unroll
    for (int s = 0; s < kSub; ++s) vv[s] = mine[(OFF + sb + s) * kRingLd];
    real ed[kSub];
    if (GIN && t0 < nx) {
      // the previous band belongs to another CTA
      if (!edge_take<real>(g_in, t0, nx, tag, gw, ed, abort_flag)) return false;
    } else if (b > 0 && t0 < nx) {
      if (!wait_progress(prog + b - 1, min(nx, t0 + kSub), abort_flag)) return false;
      // lane 0's lower neighbours (the previous band's top row) for the next
      // kSub columns, read as vectors
      const volatile typename Real4<real>::type *e4 =
          reinterpret_cast<const volatile typename Real4<real>::type *>(edge_in + t0);
#pragma unroll
      for (int q = 0; q < kSub / Real4<real>::kN; ++q) Real4<real>::unpack(e4[q], ed + q * Real4<real>::kN);
    } else {
#pragma unroll
      for (int s = 0; s < kSub; ++s) ed[s] = A.in_y;
    }
#pragma unroll
    for (int s = 0; s < kSub; ++s) {
      const int slot = (OFF + sb + s) * kRingLd;
      const typename Real2<real>::type v = vv[s];
      real down = __shfl_up_sync(kFull, psi, 1);
      if (lane == 0) down = ed[s];
      real p = fmadd(ay, down, fmadd(ax, psi, v.x)) * v.y;
      if (FIRST && t0 + s < lane) p = psi;
      psi = p;
      mine[slot].x = p;
      if (lane == 31) edge_out[t0 + s - 31] = p;
    }
    if (lane == 31) {
      __threadfence_block();
      prog[b] = min(nx, max(0, t0 + kSub - 31));
    }
    if (g_out) {
      // the unit's last band: the kSub columns of its top row finished in
      // this sub-window go to the next unit's CTA as tagged words
      __syncwarp();
      const int c = t0 - 31 + lane;
      if (lane < kSub && (unsigned)c < (unsigned)nx) {
        unsigned long long w[EdgeWords<real>::kW];
        EdgeWords<real>::encode(edge_out[c], (unsigned long long)tag << 32, w);
#pragma unroll
        for (int q = 0; q < EdgeWords<real>::kW; ++q)
          st_relaxed(g_out + (size_t)c * EdgeWords<real>::kW + q, w[q]);
      }
    }
  }
  return true;
}

// One band of 32 rows of one angle, swept by one warp.  GIN: the band below
// belongs to another CTA (the first band of a unit with an incoming edge row).
template <typename real, int NW, bool GIN>
__device__ bool sweep_band(int b, const SweepArgs<real> &A, const SweepSmem &S, const EdgeLink &L,
                           volatile int *abort_flag) {
  using real2 = typename Real2<real>::type;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  real2 *ring = reinterpret_cast<real2 *>(S.tiles) + wid * (kRing * kRingLd);
  real2 *mine = ring + lane;
  // edge rows: column u at index u + kEdgePad (columns -31 .. nx + 31 fit)
  real *edge = reinterpret_cast<real *>(S.edge);
  real *edge_out = edge + (b % (NW + 1)) * S.edge_ld + kEdgePad;
  const real *edge_in = edge + ((b + NW) % (NW + 1)) * S.edge_ld + kEdgePad;
  volatile int *prog = S.prog;
  const int nx = A.nx;
  const int nch = (nx + 31) >> 5;
  real psi = A.in_x;  // this lane's last value: the left neighbour of its next cell
  // a neighbouring band in another CTA: the unit's first band reads, its
  // last band writes, the tagged edge words
  const unsigned long long *g_in = GIN ? L.g_in : nullptr;
  unsigned long long *g_out = b == L.b0 + L.nb - 1 ? L.g_out : nullptr;
  unsigned long long gw[EdgeWords<real>::kW];
#pragma unroll
  for (int q = 0; q < EdgeWords<real>::kW; ++q) gw[q] = 0ull;
  if (GIN) edge_load<real>(g_in, 0, nx, gw);
  ChunkRegs<real> R;
  load_chunk(A, b, 0, R);
  for (int k = 0; k <= nch; ++k) {
    if (k >= 2) write_chunk(A, b, k - 2, ring);  // its slots are reused by chunk k
    __syncwarp();
    if (k < nch) stage_chunk(A, R, b, k, ring);
    __syncwarp();
    if (k + 1 < nch) load_chunk(A, b, k + 1, R);  // in flight during the steps below
    bool ok;
    if (k == 0)
      ok = sweep_window<real, NW, 0, true, GIN>(b, k, A, mine, psi, edge_in, edge_out, prog,
                                                   abort_flag, g_in, g_out, L.tag, gw);
    else if (k & 1)
      ok = sweep_window<real, NW, 32, false, GIN>(b, k, A, mine, psi, edge_in, edge_out, prog,
                                                   abort_flag, g_in, g_out, L.tag, gw);
    else
      ok = sweep_window<real, NW, 0, false, GIN>(b, k, A, mine, psi, edge_in, edge_out, prog,
                                                   abort_flag, g_in, g_out, L.tag, gw);
    if (!ok) return false;
  }
  __syncwarp();
  write_chunk(A, b, nch - 1, ring);
  __syncwarp();
  return true;
}

// Bands b0 .. b0 + nb - 1 of one angle by one CTA: warp w sweeps bands
// b0 + w, b0 + w + NW, ...  Returns, in every thread of the CTA, false if a
// wait of any warp gave up (a per-warp result would split the CTA between
// the caller's branches).
template <typename real, int NW>
__device__ bool sweep_unit(const SweepArgs<real> &A, const SweepSmem &S, const EdgeLink &L,
                           volatile int *abort_flag) {
  __syncthreads();
  for (int i = L.b0 + threadIdx.x; i < L.b0 + L.nb; i += blockDim.x) S.prog[i] = 0;
  __syncthreads();
  bool ok = true;
  const int wid = threadIdx.x >> 5;
  for (int b = L.b0 + wid; b < L.b0 + L.nb && ok; b += NW) {
    const bool gin = b == L.b0 && L.g_in;
    ok = gin ? sweep_band<real, NW, true>(b, A, S, L, abort_flag)
             : sweep_band<real, NW, false>(b, A, S, L, abort_flag);
  }
  if (!ok) *abort_flag = 1;
  return __syncthreads_and(ok) != 0;
}

template <typename real>
__device__ SweepArgs<real> unit_args(const Inst &I, int j) {
  SweepArgs<real> A;
  const int k = I.idx[j];
  const double ox = I.ox[k], oy = I.oy[k];
  A.nx = I.nx;
  A.ny = I.ny;
  A.flipx = ox < 0;
  A.flipy = oy < 0;
  A.ax = real(fabs(ox) / I.hx);
  A.ay = real(fabs(oy) / I.hy);
  A.in_x = real(ox > 0 ? I.psi_edge[0] : (ox < 0 ? I.psi_edge[1] : 0.0));
  A.in_y = real(oy > 0 ? I.psi_edge[2] : (oy < 0 ? I.psi_edge[3] : 0.0));
  if (I.refl_base) {  // a reflective edge's inflow is in the fixed source
    if (I.reflect[ox > 0 ? 0 : 1]) A.in_x = real(0);
    if (I.reflect[oy > 0 ? 2 : 3]) A.in_y = real(0);
  }
  A.sig_t = as_c<real>(I.sig_t);
  A.src = as_c<real>(I.s0) + (size_t)I.N * j;
  A.sphi = as_c<real>(I.sphi);
  A.psi = as<real>(I.Psi) + (size_t)I.N * j;
  return A;
}


template <typename real>
__global__ void __launch_bounds__(SweepCfg<real>::NW * 32)
k_si(const Inst *__restrict__ insts, SiCtl ctl) {
  constexpr int NW = SweepCfg<real>::NW;
  extern __shared__ __align__(16) unsigned char smem[];
  using real2 = typename Real2<real>::type;
  SweepSmem S;
  S.tiles = smem;
  size_t off = (size_t)NW * kRing * kRingLd * sizeof(real2);
  S.edge = smem + off;
  off += (size_t)(NW + 1) * edge_ld(ctl.nx_max) * sizeof(real);
  S.prog = reinterpret_cast<int *>(smem + off);
  off += (size_t)(ctl.bands_max + 3) / 4 * 4 * sizeof(int);
  int *active = reinterpret_cast<int *>(smem + off);
  off += (size_t)(ctl.n_inst + 3) / 4 * 4 * sizeof(int);
  double *relax = reinterpret_cast<double *>(smem + off);  // relaxation state, 3 per instance
  off += (size_t)3 * ctl.n_inst * sizeof(double);
  double *dsa_sc = reinterpret_cast<double *>(smem + off);  // CG scalars (DSA)
  int *dsa_on = reinterpret_cast<int *>(smem + off + dsa_scalar_bytes(ctl.n_inst, ctl.any_dsa));
  off += dsa_smem_bytes(ctl.n_inst, ctl.any_dsa);
  real *gam = reinterpret_cast<real *>(smem + off);  // gam_max scalar-flux weights
  S.edge_ld = edge_ld(ctl.nx_max);
  __shared__ int unit_s, n_active_s;
  volatile int *abort_flag = ctl.abort_flag;

  for (int i = threadIdx.x; i < ctl.n_inst; i += blockDim.x) {
    active[i] = (*insts[i].status == kOk) ? 1 : 0;
    relax_reset(relax + 3 * i);
  }
  // tags of the edge words: 20 bits of the launch counter, 12 of the iteration
  const unsigned epoch_tag = (*(volatile unsigned *)ctl.epoch & 0xfffffu) << 12;
  __syncthreads();
  if (ctl.any_dsa) {
    // DSA coefficients of this step (read after the first grid barrier)
    for (int i = 0; i < ctl.n_inst; ++i)
      if (active[i] && insts[i].dsa) dsa_setup<real>(insts[i]);
  }

  for (int it = 0;; ++it) {
    if (threadIdx.x == 0) {
      int n = 0;
      for (int i = 0; i < ctl.n_inst; ++i) n += active[i];
      n_active_s = n;
    }
    __syncthreads();
    if (n_active_s == 0) break;

    // ---- phase A: sweeps of all active (instance, angle) units ----
    for (;;) {
      if (threadIdx.x == 0) unit_s = (int)atomicAdd(ctl.work + (it & 1), 1u);
      __syncthreads();
      const int u = unit_s;
      __syncthreads();
      if (u >= ctl.n_units) break;
      const SiUnit U = ctl.units[u];
      if (!active[U.inst]) continue;
      const SweepArgs<real> A = unit_args<real>(insts[U.inst], U.angle);
      EdgeLink L;
      L.b0 = U.b0;
      L.nb = U.nb;
      L.g_in = U.in_row >= 0 ? ctl.gedge + (size_t)U.in_row * ctl.gedge_ld : nullptr;
      L.g_out = U.out_row >= 0 ? ctl.gedge + (size_t)U.out_row * ctl.gedge_ld : nullptr;
      L.tag = epoch_tag | ((unsigned)(it + 1) & 0xfffu);
      if (!sweep_unit<real, NW>(A, S, L, abort_flag)) break;
    }
    if (!grid_barrier(ctl.bar, abort_flag)) break;

    // ---- phase B: phi_new = sum_j gamma_j psi_j, convergence maxima ----
    if (blockIdx.x == 0) {
      for (int i = threadIdx.x; i < ctl.n_inst; i += blockDim.x) {
        insts[i].conv[((it + 1) & 1) * 2 + 0] = 0ull;
        insts[i].conv[((it + 1) & 1) * 2 + 1] = 0ull;
      }
      if (threadIdx.x == 0) ctl.work[(it + 1) & 1] = 0u;
    }
    for (int i = 0; i < ctl.n_inst; ++i) {
      if (!active[i]) continue;
      const Inst &I = insts[i];
      const int N = I.N, r = I.r;
      const real *psi = as_c<real>(I.Psi);
      const real *ss4 = as_c<real>(I.ss4);
      const real *pold = as_c<real>((it & 1) ? I.phi1 : I.phi0);
      real *pnew = as<real>((it & 1) ? I.phi0 : I.phi1);
      real *sphi = as<real>(I.sphi);
      __syncthreads();
      for (int j = threadIdx.x; j < r; j += blockDim.x)
        gam[j] = real(I.gamma_ext ? I.gamma_ext[j] : I.small[I.lay.gamma + j]);
      __syncthreads();
      // the convergence test measures the sweeps' change phi^{l+1/2} - phi^l,
      // with or without DSA (the DSA correction multiplies rounding noise by
      // up to sigma_s / sigma_a, so phi^{l+1} - phi^l would stall above a
      // tolerance near the working precision)
      real dmax = real(0), pmax = real(0);  // |differences| and |phi| in the working precision
      if (I.dsa) {
        // phi^{l+1/2}, and the right-hand side of its DSA correction
        double rz = 0, bb = 0;
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
          real acc = real(0);
          for (int j = 0; j < r; ++j) acc = fmadd(gam[j], psi[(size_t)N * j + c], acc);
          pnew[c] = acc;
          const real po = pold[c];
          dsa_rhs<real>(I, c, acc, po, rz, bb);
          dmax = max(dmax, abs(acc - po));
          pmax = max(pmax, abs(acc));
          if (!isfinite(acc)) dmax = real(INFINITY);  // diverged (max() drops NaN)
        }
        __shared__ double red[64];
        block_sum2(rz, bb, red);
        if (threadIdx.x == 0) {
          dsa_slot(ctl, i, kDsaRz)[blockIdx.x] = rz;
          dsa_slot(ctl, i, kDsaBb)[blockIdx.x] = bb;
        }
      } else {
        const real om = real(relax[3 * i]);  // relaxation (1: the plain iteration)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
          real acc = real(0);
          for (int j = 0; j < r; ++j) acc = fmadd(gam[j], psi[(size_t)N * j + c], acc);
          const real po = pold[c];
          const real pn = om == real(1) ? acc : fmadd(om, acc - po, po);
          pnew[c] = pn;
          sphi[c] = ss4[c] * pn;
          dmax = max(dmax, abs(acc - po));
          pmax = max(pmax, abs(acc));
          if (!isfinite(acc)) dmax = real(INFINITY);  // diverged (max() drops NaN)
        }
      }
      dmax = warp_max(dmax);
      pmax = warp_max(pmax);
      if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(I.conv + (it & 1) * 2 + 0, (double)dmax);
        atomic_max_nonneg(I.conv + (it & 1) * 2 + 1, (double)pmax);
      }
      if (I.refl_base) {
        // reflective edges: the next sweeps' inflow from these sweeps
        const int ne = I.r * (I.ny + I.nx);
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x)
          refl_inject<real>(I, psi, e);
      }
    }
    if (!grid_barrier(ctl.bar, abort_flag)) break;

    if (ctl.any_dsa) {
      // ---- DSA: delta from A delta = sigma_s (phi^{l+1/2} - phi^l), then
      // phi^{l+1} = phi^{l+1/2} + delta feeds the next sweeps ----
      for (int i = threadIdx.x; i < ctl.n_inst; i += blockDim.x)
        dsa_on[i] = active[i] && insts[i].dsa;
      __syncthreads();
      if (!dsa_solve<real>(insts, ctl, dsa_on, dsa_sc, abort_flag)) break;
      for (int i = 0; i < ctl.n_inst; ++i) {
        if (!active[i] || !insts[i].dsa) continue;
        const Inst &I = insts[i];
        const int N = I.N;
        const real *ss4 = as_c<real>(I.ss4), *x = as_c<real>(I.dsa_x);
        real *pnew = as<real>((it & 1) ? I.phi0 : I.phi1);
        real *sphi = as<real>(I.sphi);
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
          const real v = pnew[c] + x[c];
          pnew[c] = v;
          sphi[c] = ss4[c] * v;
        }
      }
      if (!grid_barrier(ctl.bar, abort_flag)) break;
    }

    // ---- phase C: every CTA takes the same decision per instance ----
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < ctl.n_inst; ++i) {
        if (!active[i]) continue;
        const Inst &I = insts[i];
        volatile unsigned long long *cv = I.conv + (it & 1) * 2;
        const double d = __longlong_as_double((long long)cv[0]);
        const double m = __longlong_as_double((long long)cv[1]);
        const int done_iters = it + 1;
        bool done;
        if (ctl.force_iters > 0) {
          done = done_iters >= ctl.force_iters;
          if (done) active[i] = 0;
          continue;
        }
        // DLR only (SN: gamma = w > 0); true: diverging even when relaxed
        const bool diverged = !I.dsa && !I.gamma_ext && relax_track(d, m, relax + 3 * i);
        if (diverged || !(d <= 1.0e308)) {  // or a non-finite scalar flux
          done = true;
          if (blockIdx.x == 0) set_status(I.status, kENotConv);
        } else if (I.fixed_iters > 0) {
          done = done_iters >= I.fixed_iters;
        } else {
          done = d <= I.si_tol * m;
          if (!done && done_iters >= I.max_iter) {
            done = true;
            if (blockIdx.x == 0) set_status(I.status, kENotConv);
          }
        }
        if (done) {
          active[i] = 0;
          if (blockIdx.x == 0) {
            *I.iters = done_iters;
            atomicAdd(I.iters_total, (unsigned long long)done_iters);
          }
        }
      }
    }
    __syncthreads();
  }
  // a wait that gave up marks every still-active instance
  if (*abort_flag && blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < ctl.n_inst; ++i)
      if (active[i]) set_status(insts[i].status, kETimeout);
  }
}

// Resets the barrier, the unit counters and the convergence maxima of
// iteration 0 before each source-iteration launch.
__global__ void k_si_prep(const Inst *__restrict__ insts, int n, SiCtl ctl) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    ctl.bar[0] = 0u;
    ctl.work[0] = 0u;
    ctl.work[1] = 0u;
    *ctl.abort_flag = 0;
    *ctl.epoch += 1u;  // stale edge words of earlier launches never match
  }
  if (t < n) {
    insts[t].conv[0] = 0ull;
    insts[t].conv[1] = 0ull;
    *insts[t].nonpos = 0;
  }
}

// Standalone sweeps (dlr_sweep): one CTA per direction.
template <typename real>
__global__ void __launch_bounds__(SweepCfg<real>::NW * 32)
k_sweep_dirs(int nx, int ny, double hx, double hy, const double *dirs,
             const double *psi_edge, const real *sig_t, const real *src, real *psi,
             int nx_max, int *abort_flag) {
  constexpr int NW = SweepCfg<real>::NW;
  extern __shared__ __align__(16) unsigned char smem[];
  using real2 = typename Real2<real>::type;
  SweepSmem S;
  S.tiles = smem;
  size_t off = (size_t)NW * kRing * kRingLd * sizeof(real2);
  S.edge = smem + off;
  off += (size_t)(NW + 1) * edge_ld(nx_max) * sizeof(real);
  S.prog = reinterpret_cast<int *>(smem + off);
  S.edge_ld = edge_ld(nx_max);
  const int d = blockIdx.x;
  const double ox = dirs[2 * d], oy = dirs[2 * d + 1];
  SweepArgs<real> A;
  A.nx = nx;
  A.ny = ny;
  A.flipx = ox < 0;
  A.flipy = oy < 0;
  A.ax = real(fabs(ox) / hx);
  A.ay = real(fabs(oy) / hy);
  A.in_x = real(ox > 0 ? psi_edge[0] : (ox < 0 ? psi_edge[1] : 0.0));
  A.in_y = real(oy > 0 ? psi_edge[2] : (oy < 0 ? psi_edge[3] : 0.0));
  A.sig_t = sig_t;
  A.src = src + (size_t)nx * ny * d;
  A.sphi = nullptr;
  A.psi = psi + (size_t)nx * ny * d;
  EdgeLink L{};
  L.b0 = 0;
  L.nb = (ny + 31) >> 5;
  sweep_unit<real, NW>(A, S, L, abort_flag);
}

// ------------------------------------------------------------------
// host-side launch helpers
// ------------------------------------------------------------------

cudaError_t launch_si_prep(const Inst *d, int n, SiCtl ctl, cudaStream_t st) {
  return launch_pdl(k_si_prep, dim3((n + 255) / 256), dim3(256), 0, st, d, n, ctl);
}

template <typename real>
size_t si_smem_bytes(int nx_max, int bands_max, int n_inst, int gam_max, int dsa) {
  constexpr int NW = SweepCfg<real>::NW;
  using real2 = typename Real2<real>::type;
  return (size_t)NW * kRing * kRingLd * sizeof(real2) + (size_t)(NW + 1) * edge_ld(nx_max) * sizeof(real) +
         (size_t)(bands_max + 3) / 4 * 4 * sizeof(int) + (size_t)(n_inst + 3) / 4 * 4 * sizeof(int) +
         (size_t)3 * n_inst * sizeof(double) + dsa_smem_bytes(n_inst, dsa) + (size_t)gam_max * sizeof(real);
}

template <typename real>
cudaError_t launch_si(const Inst *d_insts, const SiCtl &ctl, int grid, cudaStream_t st) {
  constexpr int NW = SweepCfg<real>::NW;
  size_t smem = si_smem_bytes<real>(ctl.nx_max, ctl.bands_max, ctl.n_inst, ctl.gam_max, ctl.any_dsa);
  cudaError_t e = cudaFuncSetAttribute(k_si<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NW * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_si<real>, d_insts, ctl);
}

template <typename real>
int si_max_grid(int nx_max, int bands_max, int n_inst, int gam_max, int dsa) {
  constexpr int NW = SweepCfg<real>::NW;
  size_t smem = si_smem_bytes<real>(nx_max, bands_max, n_inst, gam_max, dsa);
  if (cudaFuncSetAttribute(k_si<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_si<real>, NW * 32, smem) !=
      cudaSuccess)
    return 0;
  return per_sm * sms;
}

template <typename real>
cudaError_t launch_sweep_dirs(int nx, int ny, double hx, double hy, int n_dir,
                              const double *d_dirs, const double *d_edge, const real *sig_t,
                              const real *src, real *psi, int *d_abort, cudaStream_t st) {
  constexpr int NW = SweepCfg<real>::NW;
  const int bands = (ny + 31) / 32;
  size_t smem = si_smem_bytes<real>(nx, bands, 0, 0, 0);
  cudaError_t e = cudaFuncSetAttribute(k_sweep_dirs<real>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_sweep_dirs<real><<<n_dir, NW * 32, smem, st>>>(nx, ny, hx, hy, d_dirs, d_edge, sig_t, src,
                                                   psi, nx, d_abort);
  return cudaGetLastError();
}

int si_sweep_warps(bool mixed) { return mixed ? SweepCfg<float>::NW : SweepCfg<double>::NW; }
int si_sweep_lag(bool mixed) { return 32 + (mixed ? SweepCfg<float>::kSub : SweepCfg<double>::kSub); }

template size_t si_smem_bytes<float>(int, int, int, int, int);
template size_t si_smem_bytes<double>(int, int, int, int, int);
template cudaError_t launch_si<float>(const Inst *, const SiCtl &, int, cudaStream_t);
template cudaError_t launch_si<double>(const Inst *, const SiCtl &, int, cudaStream_t);
template int si_max_grid<float>(int, int, int, int, int);
template int si_max_grid<double>(int, int, int, int, int);
template cudaError_t launch_sweep_dirs<float>(int, int, double, double, int, const double *,
                                              const double *, const float *, const float *,
                                              float *, int *, cudaStream_t);
template cudaError_t launch_sweep_dirs<double>(int, int, double, double, int, const double *,
                                               const double *, const double *, const double *,
                                               double *, int *, cudaStream_t);

}  // namespace dlr
