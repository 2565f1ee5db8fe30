// Convective flux kernels: hybrid central / WENO, one direction at a time.
//
// Paper Sec. 2: the convective terms use the energy-preserving split
// (skew-symmetric) form written as numerical fluxes (Pirozzoli, JCP 2010)
// in smooth regions and, at interfaces flagged by the Ducros-type sensor, a
// WENO reconstruction of characteristic fluxes (Lax-Friedrichs splitting)
// projected back on the right eigenvectors.  These are the euler_{x,y,z}
// kernels of Table 2.  The paper's transposition kernel for x is not needed:
// every direction stages its pencils through shared memory.
//
// k_flux<DIR>  tiles of L points along DIR times W pencils (one tile per CTA
// in double precision; a persistent grid walking the tiles in single
// precision):
//   1. the tile plus GH ghost points each side arrives by TMA, one box per
//      staged field (rho, u, v, w, H, p, and the sensor test for WENO),
//      completing on an mbarrier; single precision prefetches the next
//      tiles into further buffers while computing this one;
//   2. per position a the weighted pair mass fluxes of the pairs (a, a+l),
//      l = 1..NP: m_l(a) = (a_l/4) (rho_a+rho_b)(un_a+un_b);
//   3. the central flux difference D(a) = F_{a+1/2} - F_{a-1/2} of the
//      split-form interface flux.  The pair flux of field phi is
//      m_l(a) (phi_a + phi_{a+l}), and the difference telescopes to
//        D_rho = 2 M,  M = sum_l [m_l(a) - m_l(a-l)],
//        D_phi = phi_a M + sum_l [m_l(a) phi_{a+l} - m_l(a-l) phi_{a-l}]
//      (phi = u, v, w, H; plus sum_l a_l (p_{a+l} - p_{a-l}) on the normal
//      momentum): two fused multiply-adds per field and pair instead of a
//      pair product, a difference and a multiply-add.  -scale D goes into
//      the RHS;
//   4. interface flags (max sensor over the WENO stencil > threshold, from
//      the per-point tests theta > threshold) are stored and the flagged
//      interfaces appended to a global list.
// k_weno<DIR>  one thread per listed interface (globally compacted, so
//   shocks cause no divergence in the central kernel and no idle lanes
//   here): F_weno - F_central at the interface.
// The corrections are added per point, in a fixed order, by the viscous
// kernel (or k_apply when inviscid): deterministic, no atomics on the RHS.
// Every kernel is instantiated for R = double (FP64 path) and R = float
// (arithmetic of the mixed path).
#include <string.h>

#include "s2_internal.cuh"

namespace s2 {
namespace {

// Central first-derivative coefficients a_l of order 2 NP (l = 1..NP): the
// split-form flux of order 2 NP uses the same weights (Pirozzoli 2010).
template <int NP>
__device__ __forceinline__ constexpr double acoef(int l) {
  if constexpr (NP == 1) return 1.0 / 2.0;
  else if constexpr (NP == 2) return l == 1 ? 2.0 / 3.0 : -1.0 / 12.0;
  else if constexpr (NP == 3) return l == 1 ? 3.0 / 4.0 : (l == 2 ? -3.0 / 20.0 : 1.0 / 60.0);
  else return l == 1 ? 4.0 / 5.0 : (l == 2 ? -1.0 / 5.0 : (l == 3 ? 4.0 / 105.0 : -1.0 / 280.0));
}

// Tile shapes (L points along the direction x W pencils, 256 threads):
// variant 0 is the default; variant 1 is narrower along the direction for
// small boxes.  The autotuner picks one per direction and grid.
template <int DIR, int V>
struct Tile;
template <>
struct Tile<0, 0> {  // x: 64 along x, 4 rows (y)
  static constexpr int L = 64, W = 4;
};
template <>
struct Tile<0, 1> {  // x: 32 along x, 8 rows
  static constexpr int L = 32, W = 8;
};
template <>
struct Tile<1, 0> {  // y: 32 along y, 8 columns (x)
  static constexpr int L = 32, W = 8;
};
template <>
struct Tile<1, 1> {  // y: 16 along y, 16 columns
  static constexpr int L = 16, W = 16;
};
template <>
struct Tile<2, 0> {  // z: 32 along z, 8 columns (x)
  static constexpr int L = 32, W = 8;
};
template <>
struct Tile<2, 1> {  // z: 16 along z, 16 columns
  static constexpr int L = 16, W = 16;
};
// Variant 2: the default tile with the KEEP central flux (a separate
// instantiation keeps the split-form kernels' register allocation).
template <int DIR>
struct Tile<DIR, 2> : Tile<DIR, 0> {};

constexpr int NTHREADS = 256;
constexpr int WENO_NT = 64;  // threads per CTA of the WENO kernels
enum { F_RHO = 0, F_U, F_V, F_W, F_H, F_P, F_S, NF };

// The tile a kernel of arithmetic type R works on.  Double precision uses
// the shapes above, one point per thread.  Single precision gives each
// thread PPT = 2 points along the direction (half the per-tile overhead
// per point) and, for y and z, twice the pencils across (64-byte rows in
// place of 32-byte ones per box row).
template <int DIR, int TV, class R>
struct TileR {
  static constexpr int PPT = sizeof(R) == 4 ? 2 : 1;
  static constexpr int L = Tile<DIR, TV>::L * (sizeof(R) == 4 && DIR == 0 ? 2 : 1);
  static constexpr int W = Tile<DIR, TV>::W * (sizeof(R) == 4 && DIR != 0 ? 2 : 1);
};

// Tiles of a direction: (n0, n1, n2) along the grid dimensions of the
// tiling, tile t = (t0, t1, t2) with t0 fastest.
template <int DIR, int TV, class R>
struct TileGrid {
  static constexpr int L = TileR<DIR, TV, R>::L, W = TileR<DIR, TV, R>::W;
  int n0, n1, n2;
  FastDiv f0, f1;  // divisions by n0 and n1 (set on the host)
  __host__ TileGrid(const Dev &d) {
    if (DIR == 0) { n0 = (d.nx + L - 1) / L; n1 = (d.ny + W - 1) / W; n2 = d.nz; }
    if (DIR == 1) { n0 = (d.nx + W - 1) / W; n1 = (d.ny + L - 1) / L; n2 = d.nz; }
    if (DIR == 2) { n0 = (d.nx + W - 1) / W; n1 = (d.nz + L - 1) / L; n2 = d.ny; }
    f0.init((unsigned)n0);
    f1.init((unsigned)n1);
  }
  __host__ __device__ int count() const { return n0 * n1 * n2; }
  // first interior point of the tile along (x, y, z)
  __device__ __forceinline__ void origin(int t, int &x0, int &y0, int &z0) const {
    const unsigned r = f0.div((unsigned)t), t2 = f1.div(r);
    const int t0 = t - (int)r * n0, t1 = (int)r - (int)t2 * n1;
    if (DIR == 0) { x0 = t0 * L; y0 = t1 * W; z0 = (int)t2; }
    if (DIR == 1) { x0 = t0 * W; y0 = t1 * L; z0 = (int)t2; }
    if (DIR == 2) { x0 = t0 * W; z0 = t1 * L; y0 = (int)t2; }
  }
};

// Any of the per-point sensor tests (1.0 / 0.0) of the WENO stencil
// a - WR + 1 .. a + WR of interface a + 1/2 (S points at position a),
// ORed on the integer pipe.
template <int WR, int SA, class R>
__device__ __forceinline__ bool window_any(const R *S) {
  decltype(order_bits(R(0))) any = 0;
#pragma unroll
  for (int m = 1 - WR; m <= WR; ++m) any |= order_bits(S[m * SA]);
  return any != 0;
}

template <int DIR, class R, int TV>
struct FluxLayout {
  static constexpr int L = TileR<DIR, TV, R>::L, W = TileR<DIR, TV, R>::W;
  static constexpr int PPT = TileR<DIR, TV, R>::PPT;
  static constexpr int LE = L + 2 * GH;                          // extended positions per pencil
  static constexpr int SF = LE * W;                              // words per staged field (one box)
  static constexpr int SFA = (SF * (int)sizeof(R) + 127) / 128 * 128 / (int)sizeof(R);  // 128-B aligned
  static constexpr int BAR_BYTES = 128;                          // mbarriers, padded
  // staging buffers: single precision prefetches two tiles ahead in x and
  // one in y and z (larger tiles); double precision runs one tile per CTA
  // and stages it once
  static constexpr int NBUF = sizeof(R) == 4 ? (DIR == 0 ? 3 : 2) : 1;
};

// Dynamic shared memory of a flux CTA: barriers, staging buffers and the
// pair fluxes (one mass flux per pair for the split form, the five
// components of the two-point flux for KEEP).
template <int DIR, bool HASW, class R, int TV, int NP>
constexpr size_t flux_smem(bool keep = false) {
  using Ly = FluxLayout<DIR, R, TV>;
  constexpr int NFLD = HASW ? 7 : 6;
  return Ly::BAR_BYTES +
         sizeof(R) * ((size_t)Ly::NBUF * NFLD * Ly::SFA + (size_t)(keep ? 5 : 1) * NP * (Ly::L + NP) * Ly::W);
}

// KEEP pair fluxes of a staged tile: P_l(a) = a_l f*(a, a+l), the five
// components per pair, a = -NP .. L-1 (TP[(l-1) 5 + c][position, pencil]).
template <int DIR, class R, int NP, int LT, int W, int SA, int SCS, int SCT, int SFA>
__device__ __forceinline__ void keep_pairs_tile(const R *S, R *TP, R gm1, int n) {
  constexpr int ST = LT * W;
  for (int idx = threadIdx.x; idx < ST; idx += NTHREADS) {
    int a, cc;
    if (DIR == 0) { a = idx % LT; cc = idx / LT; }
    else { a = idx / W; cc = idx % W; }
    const int q0 = (a - NP + GH) * SA + cc * SCS;
    const R ra = S[F_RHO * SFA + q0], ua = S[F_U * SFA + q0], va = S[F_V * SFA + q0];
    const R wa = S[F_W * SFA + q0], pa = S[F_P * SFA + q0];
#pragma unroll
    for (int l = 1; l <= NP; ++l) {
      const int q1 = q0 + l * SA;
      R f[5];
      keep_pair<DIR, R>(ra, ua, va, wa, pa, S[F_RHO * SFA + q1], S[F_U * SFA + q1], S[F_V * SFA + q1],
                        S[F_W * SFA + q1], S[F_P * SFA + q1], gm1, n, f);
#pragma unroll
      for (int c = 0; c < 5; ++c) TP[((l - 1) * 5 + c) * ST + a * SA + cc * SCT] = R(acoef<NP>(l)) * f[c];
    }
  }
}

// CTAs walk the tiles of a direction (t = block index, + grid extent, ...).
// With NBUF staging buffers, the tensor memory accelerator fills the
// buffers of the next NBUF - 1 tiles while tile t is computed, so the HBM
// reads of later tiles overlap the arithmetic of the current one.
template <int DIR, bool HASW, class R, int TV, int NP>
__device__ __forceinline__ void flux_body(const FluxMaps &maps, const Dev &__restrict__ d, const TileGrid<DIR, TV, R> &tg,
                                          int accumulate, const Blk &B) {
  using Ly = FluxLayout<DIR, R, TV>;
  constexpr int L = Ly::L, W = Ly::W, LE = Ly::LE, SF = Ly::SF, SFA = Ly::SFA, NBUF = Ly::NBUF, PPT = Ly::PPT;
  constexpr int LP = L / PPT;          // positions per pass of the CTA's threads
  constexpr int LT = L + NP;           // pair-flux positions a = -NP .. L-1
  constexpr int ST = LT * W;           // words per pair mass-flux slot
  constexpr int NFLD = HASW ? NF : F_S;  // the sensor is staged only for WENO
  constexpr unsigned TILE_BYTES = (unsigned)(NFLD * SF * sizeof(R));
  // Shared layouts (as the boxes land): for x the position index runs
  // fastest (threads walk along x, as the global rows do); for y and z the
  // pencil index runs fastest (threads walk across x).  Either way
  // consecutive threads touch consecutive words: no bank conflicts.
  constexpr int SA = DIR == 0 ? 1 : W;    // stride between positions
  constexpr int SCS = DIR == 0 ? LE : 1;  // stride between pencils in S
  constexpr int SCT = DIR == 0 ? LT : 1;  // stride between pencils in TP
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long *bar = (unsigned long long *)smem_raw;      // [NBUF]
  R *Sbuf = (R *)(smem_raw + Ly::BAR_BYTES);                    // [NBUF][NFLD][SFA]
  R *TP = Sbuf + NBUF * NFLD * SFA;                             // [NP][positions x pencils]
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  const int ntiles = tg.count();

  const int tid = threadIdx.x;
  const int n = DIR == 0 ? d.nx : (DIR == 1 ? d.ny : d.nz);
  const int nac = DIR == 0 ? d.ny : d.nx;   // extent across

  // box origin of a tile in padded coordinates (interior point i sits at i + GH)
  auto issue = [&](int t, int buf) {
    int x0, y0, z0;
    tg.origin(t, x0, y0, z0);
    int bx = DIR == 0 ? x0 : x0 + GH, by = DIR == 1 ? y0 : y0 + GH, bz = DIR == 2 ? z0 : z0 + GH;
    mbar_expect_tx(&bar[buf], TILE_BYTES + d.tx_extra);
#pragma unroll
    for (int f = 0; f < NFLD; ++f) tma_load_3d(Sbuf + (buf * NFLD + f) * SFA, &maps.m[f], bx, by, bz, &bar[buf]);
  };
  // tile of this CTA's iteration it, its buffer and that buffer's use count
  const int G = (int)B.nx;
  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int j = 0; j < NBUF - 1; ++j)
      if ((int)B.x + j * G < ntiles) issue((int)B.x + j * G, j);
  }
  __syncthreads();

  int it = 0;
  for (int t = (int)B.x; t < ntiles; t += G, ++it) {
    const int buf = it % NBUF;
    // the buffer of tile it + NBUF - 1 was released by the barrier that
    // ended the previous tile
    if (tid == 0 && t + (NBUF - 1) * G < ntiles) issue(t + (NBUF - 1) * G, (it + NBUF - 1) % NBUF);
    int x0, y0, z0;
    tg.origin(t, x0, y0, z0);
    const int s0 = DIR == 0 ? x0 : (DIR == 1 ? y0 : z0);
    const int c0 = DIR == 0 ? y0 : x0;
    // this thread's points (ta[p], tc) and, for y and z, their RHS so far
    // (loaded while the tile is in flight)
    int ta[PPT], tc;
    if (DIR == 0) { ta[0] = tid % LP; tc = tid / LP; }
    else { tc = tid % W; ta[0] = tid / W; }
#pragma unroll
    for (int pp = 1; pp < PPT; ++pp) ta[pp] = ta[0] + pp * LP;
    bool mine[PPT];
    long long q[PPT];
    R prev[PPT][5];
#pragma unroll
    for (int pp = 0; pp < PPT; ++pp) {
      mine[pp] = (c0 + tc < nac) && (s0 + ta[pp] < n);
      const int pi = DIR == 0 ? x0 + ta[pp] : x0 + tc;
      const int pj = DIR == 0 ? y0 + tc : (DIR == 1 ? y0 + ta[pp] : y0);
      const int pk = DIR == 2 ? z0 + ta[pp] : z0;
      // interior index in 32-bit arithmetic (n < 2^31; unused when not mine)
      q[pp] = (long long)(((unsigned)pk * (unsigned)d.ny + (unsigned)pj) * (unsigned)d.nx + (unsigned)pi);
      if (mine[pp] && !S2_OK_IDX(d, q[pp], d.n)) mine[pp] = false;
#pragma unroll
      for (int f = 0; f < 5; ++f) prev[pp][f] = (mine[pp] && accumulate) ? V.fl[f * d.n + q[pp]] : R(0);
    }
    bool late = false;
    if (tid == 0) late = !mbar_wait_bounded(&bar[buf], (unsigned)(it / NBUF) & 1u, d.wait_ns);
    if (__syncthreads_or(late)) {
      if (tid == 0) {
        atomicOr(&d.scal->status, ERR_TIMEOUT);
        // let the copies already issued for the next tiles land (bounded)
        for (int j = 1; j < NBUF; ++j)
          if (t + j * G < ntiles) mbar_wait_bounded(&bar[(it + j) % NBUF], (unsigned)((it + j) / NBUF) & 1u, d.wait_ns);
      }
      return;
    }
    const R *S = Sbuf + buf * NFLD * SFA;
    static_assert(SFA >= SF, "staging layout");

    // ---- 2. weighted pair mass fluxes m_l(a), a = -NP .. L-1 ----
    // (KEEP: the five components of a_l f*(a, a+l) instead)
    if constexpr (TV == 2) {
      keep_pairs_tile<DIR, R, NP, LT, W, SA, SCS, SCT, SFA>(S, TP, K.gamma - R(1), d.keep);
    } else
    for (int idx = tid; idx < ST; idx += NTHREADS) {
      int a, cc;                            // a in 0..LT-1 <-> position a-NP
      if (DIR == 0) { a = idx % LT; cc = idx / LT; }
      else { a = idx / W; cc = idx % W; }
      int ae = a - NP + GH;                 // extended index of the position
      const R *Sr = S + F_RHO * SFA, *Sn = S + (F_U + DIR) * SFA;
      int q0 = ae * SA + cc * SCS;
      R r0 = Sr[q0], n0 = Sn[q0];
#pragma unroll
      for (int l = 1; l <= NP; ++l) {
        int q1 = q0 + l * SA;
        TP[(l - 1) * ST + a * SA + cc * SCT] = R(0.25 * acoef<NP>(l)) * ((r0 + Sr[q1]) * (n0 + Sn[q1]));
      }
    }

    // ---- 4. flags of the interfaces this tile owns, global list ----
    // A tile owns the interfaces a+1/2 with a in 0..L-1, the first tile of a
    // pencil also the one before its first point (a = -1): every interface
    // slot 0..n of a pencil is owned exactly once.  The WENO stencil of
    // interface a+1/2 spans a-r+1 .. a+r (r = (order+1)/2).
    if constexpr (HASW) {
      const R *Ss = S + F_S * SFA;
      const int wr = (d.weno + 1) / 2;
      constexpr int NI = (L + 1) * W;
      unsigned long long mycount = 0;
      for (int base = 0; base < NI; base += NTHREADS) {
        int idx = base + tid;
        bool flag = false;
        unsigned slot = 0;
        if (idx < NI) {
          int a, cc;
          if (DIR == 0) { a = idx % (L + 1) - 1; cc = idx / (L + 1); }
          else { a = idx / W - 1; cc = idx % W; }
          int s = s0 + a;
          bool own = (c0 + cc < nac) && s <= n - 1 && (a >= 0 || s == -1);
          if (own) {
            // the stored per-point tests theta > thr are 1.0 or 0.0: the
            // interface is flagged when any point of the stencil has it
            // (max theta over the stencil > thr), ORed on the integer pipe
            const R *Sw = Ss + (a + GH) * SA + cc * SCS;
            switch (wr) {
              case 1: flag = window_any<1, SA>(Sw); break;
              case 2: flag = window_any<2, SA>(Sw); break;
              case 3: flag = window_any<3, SA>(Sw); break;
              default: flag = window_any<4, SA>(Sw); break;
            }
            if (flag && a >= 0) mycount++;
            int i = DIR == 0 ? 0 : x0 + cc, j = DIR == 0 ? y0 + cc : (DIR == 1 ? 0 : y0), k = DIR == 2 ? 0 : z0;
            slot = islot32(d, DIR, s, i, j, k);
            if (!S2_OK_IDX(d, slot, d.nslot[DIR])) flag = false;
            else d.flag[DIR][slot] = flag;
          }
        }
        unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (bal) {
          int lane = tid & 31;
          int leader = __ffs(bal) - 1;
          unsigned off = 0;
          if (lane == leader) off = atomicAdd(&d.scal->nlist[DIR], (unsigned)__popc(bal));
          off = __shfl_sync(0xffffffffu, off, leader);
          const long long at = (long long)off + __popc(bal & ((1u << lane) - 1u));
          if (flag && S2_OK_IDX(d, at, d.nslot[DIR])) d.wlist[DIR][at] = (unsigned)slot;
        }
      }
      for (int o = 16; o > 0; o >>= 1) mycount += __shfl_xor_sync(0xffffffffu, mycount, o);
      if ((tid & 31) == 0 && mycount) atomicAdd(&d.scal->wcount, mycount);
    }
    __syncthreads();

    // ---- 3. central flux difference of the thread's points -> RHS ----
    if constexpr (TV == 2) {
      // KEEP: D = 2 sum_l [P_l(a) - P_l(a-l)], P_l the stored a_l f*
#pragma unroll
      for (int pp = 0; pp < PPT; ++pp) {
        if (!mine[pp]) continue;
        const int at = (ta[pp] + NP) * SA + tc * SCT;
        const int pj = DIR == 0 ? y0 + tc : (DIR == 1 ? y0 + ta[pp] : y0);
        if (DIR == 1 && !S2_OK_IDX(d, pj, d.ny)) continue;
        const R scale2 = DIR == 0 ? K.idx2 : (DIR == 1 ? R(2) * __ldg(V.eta_y + pj) : K.idz2);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          R Dc = R(0);
#pragma unroll
          for (int l = 1; l <= NP; ++l) Dc += TP[((l - 1) * 5 + c) * ST + at] - TP[((l - 1) * 5 + c) * ST + at - l * SA];
          V.fl[c * d.n + q[pp]] = fma(-scale2, Dc, prev[pp][c]);
        }
      }
      __syncthreads();  // staging buffer and TP free for the next tile
      continue;
    }
#pragma unroll
    for (int pp = 0; pp < PPT; ++pp) {
      if (!mine[pp]) continue;
      R D[5];
      const int at = (ta[pp] + NP) * SA + tc * SCT;
      const int ap = (ta[pp] + GH) * SA + tc * SCS;
      R mp[NP], mm[NP];                     // m_l(a), m_l(a-l)
      R M = R(0);
#pragma unroll
      for (int l = 1; l <= NP; ++l) {
        mp[l - 1] = TP[(l - 1) * ST + at];
        mm[l - 1] = TP[(l - 1) * ST + at - l * SA];
        M += mp[l - 1] - mm[l - 1];
      }
      // D_rho = 2 M: in x and z the factor 2 rides on the constant scale
      // (2/dx, 2/dz, exact), saving a double-precision operation
      D[0] = DIR == 1 ? R(2) * M : M;
#pragma unroll
      for (int f = 1; f < 5; ++f) {
        const R *Sf = S + f * SFA;         // F_U .. F_H follow F_RHO
        R acc = Sf[ap] * M;
#pragma unroll
        for (int l = 1; l <= NP; ++l) {
          acc = fma(mp[l - 1], Sf[ap + l * SA], acc);
          acc = fma(-mm[l - 1], Sf[ap - l * SA], acc);
        }
        D[f] = acc;
      }
      const R *Sp = S + F_P * SFA;
      R dp = R(0);
#pragma unroll
      for (int l = 1; l <= NP; ++l) dp = fma(R(acoef<NP>(l)), Sp[ap + l * SA] - Sp[ap - l * SA], dp);
      D[1 + DIR] += dp;
      const int pj = DIR == 0 ? y0 + tc : (DIR == 1 ? y0 + ta[pp] : y0);
      if (DIR == 1 && !S2_OK_IDX(d, pj, d.ny)) continue;
      R scale = DIR == 0 ? K.idx : (DIR == 1 ? __ldg(V.eta_y + pj) : K.idz);
      const R scale0 = DIR == 0 ? K.idx2 : (DIR == 1 ? scale : K.idz2);
      V.fl[q[pp]] = fma(-scale0, D[0], prev[pp][0]);
#pragma unroll
      for (int f = 1; f < 5; ++f) V.fl[f * d.n + q[pp]] = fma(-scale, D[f], prev[pp][f]);
    }
    __syncthreads();  // staging buffer and TP free for the next tile
  }
}

template <int DIR, bool HASW, class R, int TV, int NP>
__global__ void __launch_bounds__(NTHREADS, 4) k_flux(const __grid_constant__ FluxMaps maps, Dev d,
                                                      const TileGrid<DIR, TV, R> tg, int accumulate) {
  flux_body<DIR, HASW, R, TV, NP>(maps, d, tg, accumulate, grid_blk());
}

// Batched: box b's tiles with its tensor maps maps[b] (device memory,
// 64-byte aligned) and tile grid tgs[b].
template <int DIR, bool HASW, class R, int TV, int NP>
__global__ void __launch_bounds__(NTHREADS, 4) kb_flux(BatchArgs ba, const FluxMaps *maps,
                                                       const TileGrid<DIR, TV, R> *tgs, int accumulate) {
  S2_BATCH_ENTER(ba, sd, B, b);
  const TileGrid<DIR, TV, R> tg = tgs[b];
  flux_body<DIR, HASW, R, TV, NP>(maps[b], sd, tg, accumulate, B);
}

// ------------------------------------------------------------------ WENO
// Reconstruction at i+1/2 from 2r-1 values g[0..2r-2] centred on g[r-1]:
// Jiang & Shu (r=3), Balsara & Shu (r=4), alpha_k = d_k/(eps+beta_k)^2.
// The normalisation sum alpha_k q_k / sum alpha_k is evaluated with one
// reciprocal by multiplying through by prod_k (eps+beta_k)^2, and the
// substencil polynomials' common denominator (6, 12) joins that
// reciprocal.  The caller passes eps: reconstructing 2 g with eps' = 4 eps
// gives exactly twice the reconstruction of g with eps (beta is quadratic
// in g), which lets the flux splitting skip its factor 1/2.
template <class R>
__device__ __forceinline__ R recip_pos(R x) {
  return rcp_pos(x);
}

template <class R>
__device__ __forceinline__ R weno5(const R *g, R eps) {
  R q0 = R(2) * g[0] - R(7) * g[1] + R(11) * g[2];
  R q1 = -g[1] + R(5) * g[2] + R(2) * g[3];
  R q2 = R(2) * g[2] + R(5) * g[3] - g[4];
  R t, b0, b1, b2;
  t = g[0] - R(2) * g[1] + g[2]; b0 = R(13.0 / 12.0) * t * t;
  t = g[0] - R(4) * g[1] + R(3) * g[2]; b0 += R(0.25) * t * t;
  t = g[1] - R(2) * g[2] + g[3]; b1 = R(13.0 / 12.0) * t * t;
  t = g[1] - g[3]; b1 += R(0.25) * t * t;
  t = g[2] - R(2) * g[3] + g[4]; b2 = R(13.0 / 12.0) * t * t;
  t = R(3) * g[2] - R(4) * g[3] + g[4]; b2 += R(0.25) * t * t;
  R s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  s0 *= s0; s1 *= s1; s2 *= s2;
  R a0 = R(0.1) * s1 * s2, a1 = R(0.6) * s0 * s2, a2 = R(0.3) * s0 * s1;
  return (a0 * q0 + a1 * q1 + a2 * q2) * recip_pos(R(6) * (a0 + a1 + a2));
}

template <class R>
__device__ __forceinline__ R weno7(const R *g, R eps) {
  R q0 = R(-3) * g[0] + R(13) * g[1] - R(23) * g[2] + R(25) * g[3];
  R q1 = g[1] - R(5) * g[2] + R(13) * g[3] + R(3) * g[4];
  R q2 = -g[2] + R(7) * g[3] + R(7) * g[4] - g[5];
  R q3 = R(3) * g[3] + R(13) * g[4] - R(5) * g[5] + g[6];
  // smoothness indicators: 240 x the Jiang-Shu measure as sums of squares
  // of the undivided differences of each 4-point substencil
  R bk[4];
  const R c10[4] = {R(5.0 / 2.0), R(3.0 / 2.0), R(1.0 / 2.0), R(-1.0 / 2.0)};
  const R c11[4] = {R(11.0 / 6.0), R(1.0 / 3.0), R(-1.0 / 6.0), R(1.0 / 3.0)};
  const R c2[4] = {R(2), R(1), R(0), R(-1)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    R e1 = g[k + 1] - g[k];
    R e2 = g[k + 2] - R(2) * g[k + 1] + g[k];
    R e3 = g[k + 3] - R(3) * g[k + 2] + R(3) * g[k + 1] - g[k];
    R t1 = e1 + c10[k] * e2 + c11[k] * e3;
    R t2 = e2 + c2[k] * e3;
    bk[k] = R(240) * t1 * t1 + R(260) * t2 * t2 + R(781.0 / 3.0) * e3 * e3;
  }
  R s0 = eps + bk[0], s1 = eps + bk[1], s2 = eps + bk[2], s3 = eps + bk[3];
  s0 *= s0; s1 *= s1; s2 *= s2; s3 *= s3;
  R p01 = s0 * s1, p23 = s2 * s3;
  R a0 = R(1.0 / 35.0) * s1 * p23, a1 = R(12.0 / 35.0) * s0 * p23;
  R a2 = R(18.0 / 35.0) * p01 * s3, a3 = R(4.0 / 35.0) * p01 * s2;
  return (a0 * q0 + a1 * q1 + a2 * q2 + a3 * q3) * recip_pos(R(12) * (a0 + a1 + a2 + a3));
}

// Order 3: two substencils, d = (1/3, 2/3), beta_k = (undivided difference)^2.
template <class R>
__device__ __forceinline__ R weno3(const R *g, R eps) {
  R q0 = -g[0] + R(3) * g[1];
  R q1 = g[1] + g[2];
  R t0 = g[1] - g[0], t1 = g[2] - g[1];
  R s0 = eps + t0 * t0, s1 = eps + t1 * t1;
  s0 *= s0; s1 *= s1;
  R a0 = R(1.0 / 3.0) * s1, a1 = R(2.0 / 3.0) * s0;
  return (a0 * q0 + a1 * q1) * recip_pos(R(2) * (a0 + a1));
}

template <int WR, class R>
__device__ __forceinline__ R weno_rec(const R *g, R eps) {
  if constexpr (WR == 1) return g[0];  // order 1: upwind value
  else if constexpr (WR == 2) return weno3<R>(g, eps);
  else if constexpr (WR == 3) return weno5<R>(g, eps);
  else return weno7<R>(g, eps);
}

// F_weno - F_central at every listed interface of direction DIR.
//
// In the frame (normal n, tangents t1, t2) of the interface, with the Roe
// state (u_n, u_1, u_2, H~, c~), b = gamma-1, h2 = 1/(2 c~^2), the left
// eigenvector rows applied to W = (rho, m_n, m_1, m_2, E) are
//   l_0 W = A + B,  l_4 W = A - B,  l_1 W = rho - 2A,
//   l_2 W = m_1 - u_1 rho,  l_3 W = m_2 - u_2 rho,
//   A = h2 b (q~^2/2 rho - u_n m_n - u_1 m_1 - u_2 m_2 + E),
// (a thermally perfect gas: b = chi = R/c_v(T~) at the Roe temperature,
// q~^2/2 -> q~^2 - hs here and -> hs in the entropy wave's right
// eigenvector, hs = H~ - c~^2/chi; c~^2 = gamma(T~) R T~),
//   B = h2 c~ (u_n rho - m_n),
// and, with the point's flux F = u_n W + p (0, 1, 0, 0, u_n),
//   l_e F = u_n (l_e W) + p (l_e[1] + l_e[4] u_n),
// i.e. + PA - PB, + PA + PB, - 2 PA, 0, 0 for e = 0, 4, 1, 2, 3 with
// PA = p h2 b (u_n - u~_n), PB = p h2 c~.  Lax-Friedrichs: each field's
// dissipation is the largest |eigenvalue| (u_n - c, u_n, u_n + c) over the
// stencil points.  The result goes back with the right eigenvectors.
template <int DIR, int WR, class R>
__device__ __forceinline__ void weno_body(const Dev &__restrict__ d, const Blk &B) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int NP = 2 * WR;  // stencil points s-WR+1 .. s+WR
  const View<R> V = view<R>(d);
  const Consts<R> &K = consts<R>(d);
  const unsigned cnt = d.scal->nlist[DIR];
  const R *vel[3] = {V.u, V.v, V.ww};
  const R bq = K.gamma - R(1);
  for (unsigned e0 = B.x * blockDim.x + threadIdx.x; e0 < cnt; e0 += B.nx * blockDim.x) {
    if (!S2_OK_IDX(d, e0, d.nslot[DIR])) break;
    const long long slot = d.wlist[DIR][e0];
    int i = 0, j = 0, k = 0, s;
    const unsigned us = (unsigned)slot;
    if (DIR == 0) {
      unsigned t = d.fnx1.div(us), kk = d.fny.div(t);
      s = (int)(us - t * (unsigned)(d.nx + 1)) - 1;
      j = (int)(t - kk * (unsigned)d.ny);
      k = (int)kk;
      i = s;
    } else if (DIR == 1) {
      unsigned t = d.fnx.div(us), kk = d.fny1.div(t);
      i = (int)(us - t * (unsigned)d.nx);
      s = (int)(t - kk * (unsigned)(d.ny + 1)) - 1;
      k = (int)kk;
      j = s;
    } else {
      unsigned t = d.fnx.div(us), kk = d.fny.div(t);
      i = (int)(us - t * (unsigned)d.nx);
      j = (int)(t - kk * (unsigned)d.ny);
      s = (int)kk - 1;
      k = s;
    }
    const long long stride = DIR == 0 ? 1 : (DIR == 1 ? d.sy : d.sz);
    const long long p0 = pidx(d, i, j, k);  // point s of the interface s+1/2
    // the WENO stencil and the central pairs reach p0 - 3 stride .. p0 + 4 stride
    if (!(S2_OK_IDX(d, slot, d.nslot[DIR]) && S2_OK_IDX(d, p0 - 3 * stride, d.np) &&
          S2_OK_IDX(d, p0 + 4 * stride, d.np)))
      continue;

    // --- central flux at this interface (order 2 npc): split form, or KEEP
    R FC[5] = {R(0), R(0), R(0), R(0), R(0)}, fp = R(0);
    if (d.keep) {
      for (int l = 1; l <= d.npc; ++l)
        for (int m = 0; m < l; ++m) {
          const long long a = p0 - m * stride, b = p0 + (l - m) * stride;
          R f[5];
          keep_pair<DIR, R>(__ldg(V.rho + a), __ldg(V.u + a), __ldg(V.v + a), __ldg(V.ww + a), __ldg(V.p + a),
                            __ldg(V.rho + b), __ldg(V.u + b), __ldg(V.v + b), __ldg(V.ww + b), __ldg(V.p + b),
                            K.gamma - R(1), d.keep, f);
          const R al2 = R(2) * K.acen[l];
#pragma unroll
          for (int c = 0; c < 5; ++c) FC[c] = fma(al2, f[c], FC[c]);
        }
    }
#pragma unroll
    for (int l = 1; l <= 4; ++l) {
      if (l > d.npc || d.keep) break;
      R acc[5] = {R(0), R(0), R(0), R(0), R(0)}, ps = R(0);
#pragma unroll
      for (int m = 0; m < l; ++m) {
        long long a = p0 - m * stride, b = p0 + (l - m) * stride;
        R sr = __ldg(V.rho + a) + __ldg(V.rho + b);
        R su = __ldg(V.u + a) + __ldg(V.u + b), sv = __ldg(V.v + a) + __ldg(V.v + b);
        R sw = __ldg(V.ww + a) + __ldg(V.ww + b);
        R sh = __ldg(V.H + a) + __ldg(V.H + b);
        R sun = DIR == 0 ? su : (DIR == 1 ? sv : sw);
        R mm = sr * sun;
        acc[0] += mm;
        acc[1] += mm * su;
        acc[2] += mm * sv;
        acc[3] += mm * sw;
        acc[4] += mm * sh;
        ps += __ldg(V.p + a) + __ldg(V.p + b);
      }
      R al = K.acen[l];
      FC[0] += R(0.5) * al * acc[0];
#pragma unroll
      for (int f = 1; f < 5; ++f) FC[f] += R(0.25) * al * acc[f];
      fp += al * ps;
    }
    FC[1 + DIR] += fp;

    // --- Roe average of the two interface states
    const long long ia = p0, ib = p0 + stride;
    R ra = sqrt(__ldg(V.rho + ia)), rb = sqrt(__ldg(V.rho + ib));
    R inv = recip_pos(ra + rb);
    R un = (ra * __ldg(vel[DIR] + ia) + rb * __ldg(vel[DIR] + ib)) * inv;
    R ut1 = (ra * __ldg(vel[T1] + ia) + rb * __ldg(vel[T1] + ib)) * inv;
    R ut2 = (ra * __ldg(vel[T2] + ia) + rb * __ldg(vel[T2] + ib)) * inv;
    R Ht = (ra * __ldg(V.H + ia) + rb * __ldg(V.H + ib)) * inv;
    R q2 = un * un + ut1 * ut1 + ut2 * ut2;
    // chi = (1/rho) dp/de, c~^2, the entropy wave's energy entry hs and
    // the term qa of the left rows (both |u~|^2/2 for a calorically
    // perfect gas)
    R chi = bq, c2, hs = R(0.5) * q2, qa = hs;
    if (!K.tp) {
      c2 = bq * (Ht - hs);
    } else {
      // Roe temperature: h(T~) = H~ - |u~|^2/2 by Newton's method from the
      // sqrt(rho)-weighted temperature; chi = R/c_v(T~), c~^2 = (1+chi) R T~
      bool ok = true;
      const R T0 = (ra * __ldg(V.T + ia) + rb * __ldg(V.T + ib)) * inv;
      const R Tt = tp_temperature(K, Ht - hs, T0, K.R_gas, ok);
      if (!ok) atomicOr(&d.scal->status, ERR_NONFINITE);
      chi = K.R_gas * recip_pos(tp_cp(K, Tt, recip_pos(Tt)) - K.R_gas);
      c2 = (R(1) + chi) * K.R_gas * Tt;
      hs = Ht - c2 * recip_pos(chi);
      qa = q2 - hs;
    }
    R cs = sqrt(c2);
    R h2 = R(0.5) * recip_pos(c2);
    R hb = h2 * chi, hc = h2 * cs;

    // --- per stencil point: l_e W and l_e F for the five fields
    R Vv[5][NP], G[5][NP];
    R al0 = R(0), al1 = R(0), al4 = R(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      long long q = p0 + (m - WR + 1) * stride;
      R r = __ldg(V.rho + q), unm = __ldg(vel[DIR] + q);
      R u1 = __ldg(vel[T1] + q), u2 = __ldg(vel[T2] + q);
      R pm = __ldg(V.p + q), hm = __ldg(V.H + q);
      const R Tm = __ldg(V.T + q);
      R cm = sqrt(K.tp ? tp_sound2(K, Tm) : K.gR * Tm);
      R mn = r * unm, m1 = r * u1, m2 = r * u2, E = r * hm - pm;
      R A = hb * (qa * r - un * mn - ut1 * m1 - ut2 * m2 + E);
      R B = hc * (un * r - mn);
      R PA = pm * hb * (unm - un), PB = pm * hc;
      Vv[0][m] = A + B;
      Vv[1][m] = r - R(2) * A;
      Vv[2][m] = m1 - ut1 * r;
      Vv[3][m] = m2 - ut2 * r;
      Vv[4][m] = A - B;
      G[0][m] = unm * Vv[0][m] + PA - PB;
      G[1][m] = unm * Vv[1][m] - R(2) * PA;
      G[2][m] = unm * Vv[2][m];
      G[3][m] = unm * Vv[3][m];
      G[4][m] = unm * Vv[4][m] + PA + PB;
      al0 = fmax(al0, fabs(unm - cm));
      al1 = fmax(al1, fabs(unm));
      al4 = fmax(al4, fabs(unm + cm));
    }
    // Lax-Friedrichs split g+- = (G +- alpha V) / 2, reconstructed as
    // G +- alpha V with 4 eps (exactly twice the result), halved once
    R gh[5];
    const R eps4 = R(4e-6);
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      R alpha = e == 0 ? al0 : (e == 4 ? al4 : al1);
      R gp[2 * WR - 1], gmn[2 * WR - 1];
#pragma unroll
      for (int m = 0; m < 2 * WR - 1; ++m) {
        gp[m] = fma(alpha, Vv[e][m], G[e][m]);
        int mm = NP - 1 - m;
        gmn[m] = fma(-alpha, Vv[e][mm], G[e][mm]);
      }
      gh[e] = R(0.5) * (weno_rec<WR, R>(gp, eps4) + weno_rec<WR, R>(gmn, eps4));
    }
    // --- back to conserved fluxes with the right eigenvectors
    R s014 = gh[0] + gh[1] + gh[4];
    R dn = gh[4] - gh[0];
    R Fr[5];
    Fr[0] = s014;
    Fr[1 + DIR] = un * s014 + cs * dn;
    Fr[1 + T1] = ut1 * s014 + gh[2];
    Fr[1 + T2] = ut2 * s014 + gh[3];
    Fr[4] = Ht * (gh[0] + gh[4]) + un * cs * dn + hs * gh[1] + ut1 * gh[2] + ut2 * gh[3];
    const long long ns = d.nslot[DIR];
#pragma unroll
    for (int f = 0; f < 5; ++f) V.dF[DIR][f * ns + slot] = Fr[f] - FC[f];
  }
}

template <int DIR, int WR, class R>
__global__ void __launch_bounds__(WENO_NT) k_weno(Dev d) {
  weno_body<DIR, WR, R>(d, grid_blk());
}

template <int DIR, int WR, class R>
__global__ void __launch_bounds__(WENO_NT) kb_weno(BatchArgs ba) {
  S2_BATCH_ENTER(ba, sd, B, b_box);
  weno_body<DIR, WR, R>(sd, B);
}

// Single precision (bound by memory traffic): a persistent grid, as many
// CTAs as fit on the device at once, each prefetching its next two tiles.
// Double precision (bound by the double-precision unit): one tile per CTA,
// so that more CTAs at different phases share each multiprocessor and keep
// that unit busy (measured faster than the persistent loop).
template <int DIR, bool HASW, class R, int TV, int NP>
cudaError_t launch_one(const Dev &d, const FluxMaps &maps, int accumulate, cudaStream_t st) {
  static int per_sm = 0;  // resident CTAs per multiprocessor (per instantiation)
  const size_t smem = flux_smem<DIR, HASW, R, TV, NP>(TV == 2);
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_flux<DIR, HASW, R, TV, NP>, NTHREADS, smem) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    per_sm = b;
  }
  const TileGrid<DIR, TV, R> tg(d);
  const int ntiles = tg.count();
  const int cps = d.flux_cps[DIR] > 0 && d.flux_cps[DIR] < per_sm ? d.flux_cps[DIR] : per_sm;
  const int nb = sizeof(R) == 8 ? ntiles : (ntiles < cps * d.nsm ? ntiles : cps * d.nsm);
  k_flux<DIR, HASW, R, TV, NP><<<nb, NTHREADS, smem, st>>>(maps, d, tg, accumulate);
  return cudaGetLastError();
}

template <int DIR, bool HASW, class R, int TV>
cudaError_t launch_np(const Dev &d, const FluxMaps &maps, int accumulate, cudaStream_t st) {
  switch (d.npc) {
    case 1: return launch_one<DIR, HASW, R, TV, 1>(d, maps, accumulate, st);
    case 2: return launch_one<DIR, HASW, R, TV, 2>(d, maps, accumulate, st);
    case 3: return launch_one<DIR, HASW, R, TV, 3>(d, maps, accumulate, st);
    case 4: return launch_one<DIR, HASW, R, TV, 4>(d, maps, accumulate, st);
  }
  return cudaErrorInvalidValue;
}

template <int DIR, bool HASW, class R>
cudaError_t launch_tv(const Dev &d, const FluxMaps (&maps)[2], int accumulate, cudaStream_t st) {
  if (d.keep) return launch_np<DIR, HASW, R, 2>(d, maps[0], accumulate, st);  // KEEP: the default tile
  return d.tile[DIR] ? launch_np<DIR, HASW, R, 1>(d, maps[1], accumulate, st)
                     : launch_np<DIR, HASW, R, 0>(d, maps[0], accumulate, st);
}

template <int DIR, int WR, class R>
cudaError_t launch_weno_one(const Dev &d, cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // small CTAs: the flagged interfaces (a device-side count, often a few
  // per cent of the slots) then spread evenly over the multiprocessors
  long long need = (d.nslot[DIR] + WENO_NT - 1) / WENO_NT;
  long long cap = (long long)(d.weno_cps > 0 ? d.weno_cps : 16) * sms;
  unsigned nb = (unsigned)(need < cap ? need : cap);
  if (nb == 0) nb = 1;
  k_weno<DIR, WR, R><<<nb, WENO_NT, 0, st>>>(d);
  return cudaGetLastError();
}

template <int DIR, bool HASW, class R, int TV, int NP>
cudaError_t set_attr_one() {
  cudaError_t e = cudaFuncSetAttribute(k_flux<DIR, HASW, R, TV, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)flux_smem<DIR, HASW, R, TV, NP>(TV == 2));
  cudaError_t e2 = cudaFuncSetAttribute(kb_flux<DIR, HASW, R, TV, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)flux_smem<DIR, HASW, R, TV, NP>(TV == 2));
  return e != cudaSuccess ? e : e2;
}

template <int DIR, class R>
cudaError_t set_attr() {
  cudaError_t e = cudaSuccess, r;
#define S2_A(H, T, N) \
  if ((r = set_attr_one<DIR, H, R, T, N>()) != cudaSuccess) e = r;
  S2_A(false, 0, 1) S2_A(false, 0, 2) S2_A(false, 0, 3) S2_A(false, 0, 4)
  S2_A(false, 1, 1) S2_A(false, 1, 2) S2_A(false, 1, 3) S2_A(false, 1, 4)
  S2_A(true, 0, 1) S2_A(true, 0, 2) S2_A(true, 0, 3) S2_A(true, 0, 4)
  S2_A(true, 1, 1) S2_A(true, 1, 2) S2_A(true, 1, 3) S2_A(true, 1, 4)
  S2_A(false, 2, 1) S2_A(false, 2, 2) S2_A(false, 2, 3) S2_A(false, 2, 4)
  S2_A(true, 2, 1) S2_A(true, 2, 2) S2_A(true, 2, 3) S2_A(true, 2, 4)
#undef S2_A
  return e;
}

template <class R>
cudaError_t flux_dispatch(const Dev &d, const FluxMaps (&maps)[2], int dir, int accumulate, cudaStream_t st) {
  const bool w = d.weno > 0;
  switch (dir) {
    case 0: return w ? launch_tv<0, true, R>(d, maps, accumulate, st) : launch_tv<0, false, R>(d, maps, accumulate, st);
    case 1: return w ? launch_tv<1, true, R>(d, maps, accumulate, st) : launch_tv<1, false, R>(d, maps, accumulate, st);
    case 2: return w ? launch_tv<2, true, R>(d, maps, accumulate, st) : launch_tv<2, false, R>(d, maps, accumulate, st);
  }
  return cudaErrorInvalidValue;
}

// Tensor map of one padded field (extent px x py x pz, x contiguous) with
// the tile box of direction DIR, variant TV.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

template <int DIR, int TV, class R>
cudaError_t make_map(const Dev &d, void *base, CUtensorMap *out) {
  constexpr int L = TileR<DIR, TV, R>::L, W = TileR<DIR, TV, R>::W, LE = L + 2 * GH;
  constexpr bool dbl = sizeof(R) == 8;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t es = dbl ? 8 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)d.px, (cuuint64_t)d.py, (cuuint64_t)d.pz};
  cuuint64_t strides[2] = {(cuuint64_t)d.px * es, (cuuint64_t)d.px * d.py * es};
  cuuint32_t box[3];
  if (DIR == 0) { box[0] = LE; box[1] = W; box[2] = 1; }
  if (DIR == 1) { box[0] = W; box[1] = LE; box[2] = 1; }
  if (DIR == 2) { box[0] = W; box[1] = 1; box[2] = LE; }
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(out, dbl ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class R>
cudaError_t weno_dispatch(const Dev &d, int dir, cudaStream_t st) {
  const int wr = (d.weno + 1) / 2;
  switch (dir * 10 + wr) {
    case 1: return launch_weno_one<0, 1, R>(d, st);
    case 2: return launch_weno_one<0, 2, R>(d, st);
    case 3: return launch_weno_one<0, 3, R>(d, st);
    case 4: return launch_weno_one<0, 4, R>(d, st);
    case 11: return launch_weno_one<1, 1, R>(d, st);
    case 12: return launch_weno_one<1, 2, R>(d, st);
    case 13: return launch_weno_one<1, 3, R>(d, st);
    case 14: return launch_weno_one<1, 4, R>(d, st);
    case 21: return launch_weno_one<2, 1, R>(d, st);
    case 22: return launch_weno_one<2, 2, R>(d, st);
    case 23: return launch_weno_one<2, 3, R>(d, st);
    case 24: return launch_weno_one<2, 4, R>(d, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t flux_set_attributes() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_attr<0, double>()) != cudaSuccess) e = r;
  if ((r = set_attr<1, double>()) != cudaSuccess) e = r;
  if ((r = set_attr<2, double>()) != cudaSuccess) e = r;
  if ((r = set_attr<0, float>()) != cudaSuccess) e = r;
  if ((r = set_attr<1, float>()) != cudaSuccess) e = r;
  if ((r = set_attr<2, float>()) != cudaSuccess) e = r;
  return e;
}

cudaError_t launch_flux(const Dev &d, const FluxMaps (&maps)[2], int dir, int accumulate, cudaStream_t st) {
  return d.mixed ? flux_dispatch<float>(d, maps, dir, accumulate, st)
                 : flux_dispatch<double>(d, maps, dir, accumulate, st);
}

template <class R>
cudaError_t make_maps_dir(const Dev &d, void *field, int f, FluxMaps (&maps)[3][2]) {
  cudaError_t e = make_map<0, 0, R>(d, field, &maps[0][0].m[f]);
  if (e == cudaSuccess) e = make_map<0, 1, R>(d, field, &maps[0][1].m[f]);
  if (e == cudaSuccess) e = make_map<1, 0, R>(d, field, &maps[1][0].m[f]);
  if (e == cudaSuccess) e = make_map<1, 1, R>(d, field, &maps[1][1].m[f]);
  if (e == cudaSuccess) e = make_map<2, 0, R>(d, field, &maps[2][0].m[f]);
  if (e == cudaSuccess) e = make_map<2, 1, R>(d, field, &maps[2][1].m[f]);
  return e;
}

cudaError_t flux_make_maps(const Dev &d, FluxMaps (&maps)[3][2]) {
  void *fields[7] = {d.rho, d.u, d.v, d.ww, d.H, d.p, d.sens};
  const bool dbl = !d.mixed;
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < 7 && e == cudaSuccess; ++f) {
    if ((uintptr_t)fields[f] % 16) return cudaErrorInvalidValue;
    if (dbl) e = make_maps_dir<double>(d, fields[f], f, maps);
    else e = make_maps_dir<float>(d, fields[f], f, maps);
  }
  return e;
}

cudaError_t launch_weno(const Dev &d, int dir, cudaStream_t st) {
  return d.mixed ? weno_dispatch<float>(d, dir, st) : weno_dispatch<double>(d, dir, st);
}

// ------------------------------------------------------- batched launches
// The flux kernel instantiation of a Dev (precision, WENO or not, tile
// variant, central order): F::run<DIR, HASW, R, TV, NP>().
namespace {

template <class F, int DIR, bool HASW, class R, int TV>
cudaError_t sel_np(const Dev &d, F &f) {
  switch (d.npc) {
    case 1: return f.template run<DIR, HASW, R, TV, 1>();
    case 2: return f.template run<DIR, HASW, R, TV, 2>();
    case 3: return f.template run<DIR, HASW, R, TV, 3>();
    case 4: return f.template run<DIR, HASW, R, TV, 4>();
  }
  return cudaErrorInvalidValue;
}

template <class F, int DIR, class R>
cudaError_t sel_w(const Dev &d, F &f) {
  if (d.keep) return d.weno > 0 ? sel_np<F, DIR, true, R, 2>(d, f) : sel_np<F, DIR, false, R, 2>(d, f);
  if (d.weno > 0) return d.tile[DIR] ? sel_np<F, DIR, true, R, 1>(d, f) : sel_np<F, DIR, true, R, 0>(d, f);
  return d.tile[DIR] ? sel_np<F, DIR, false, R, 1>(d, f) : sel_np<F, DIR, false, R, 0>(d, f);
}

template <class F, class R>
cudaError_t sel_dir(const Dev &d, int dir, F &f) {
  switch (dir) {
    case 0: return sel_w<F, 0, R>(d, f);
    case 1: return sel_w<F, 1, R>(d, f);
    case 2: return sel_w<F, 2, R>(d, f);
  }
  return cudaErrorInvalidValue;
}

template <class F>
cudaError_t flux_select(const Dev &d, int dir, F &f) {
  return d.mixed ? sel_dir<F, float>(d, dir, f) : sel_dir<F, double>(d, dir, f);
}

struct FluxPlan {
  const Dev &d;
  FluxBoxPlan &out;
  template <int DIR, bool HASW, class R, int TV, int NP>
  cudaError_t run() {
    static int per_sm = 0;  // resident CTAs per multiprocessor of the batched kernel
    if (per_sm == 0) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kb_flux<DIR, HASW, R, TV, NP>, NTHREADS,
                                                        flux_smem<DIR, HASW, R, TV, NP>(TV == 2)) != cudaSuccess ||
          b < 1)
        b = 1;
      per_sm = b;
    }
    const TileGrid<DIR, TV, R> tg(d);
    static_assert(sizeof(tg) <= sizeof(out.tg), "tile grid record");
    memcpy(out.tg, &tg, sizeof(tg));
    out.tg_size = (int)sizeof(tg);
    out.tiles = tg.count();
    out.per_sm = d.flux_cps[DIR] > 0 && d.flux_cps[DIR] < per_sm ? d.flux_cps[DIR] : per_sm;
    out.persistent = sizeof(R) == 4;
    return cudaSuccess;
  }
};

struct FluxBatchLaunch {
  const BatchArgs &ba;
  unsigned total;
  const FluxMaps *maps;
  const void *tgs;
  int accumulate;
  cudaStream_t st;
  template <int DIR, bool HASW, class R, int TV, int NP>
  cudaError_t run() {
    kb_flux<DIR, HASW, R, TV, NP><<<total, NTHREADS, flux_smem<DIR, HASW, R, TV, NP>(TV == 2), st>>>(
        ba, maps, (const TileGrid<DIR, TV, R> *)tgs, accumulate);
    return cudaGetLastError();
  }
};

template <int DIR, class R>
cudaError_t weno_batch_wr(const Dev &d0, const BatchArgs &ba, unsigned total, cudaStream_t st) {
  switch ((d0.weno + 1) / 2) {
    case 1: kb_weno<DIR, 1, R><<<total, WENO_NT, 0, st>>>(ba); break;
    case 2: kb_weno<DIR, 2, R><<<total, WENO_NT, 0, st>>>(ba); break;
    case 3: kb_weno<DIR, 3, R><<<total, WENO_NT, 0, st>>>(ba); break;
    case 4: kb_weno<DIR, 4, R><<<total, WENO_NT, 0, st>>>(ba); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t weno_batch_dir(const Dev &d0, const BatchArgs &ba, unsigned total, int dir, cudaStream_t st) {
  switch (dir) {
    case 0: return weno_batch_wr<0, R>(d0, ba, total, st);
    case 1: return weno_batch_wr<1, R>(d0, ba, total, st);
    case 2: return weno_batch_wr<2, R>(d0, ba, total, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t flux_batch_plan(const Dev &d, int dir, FluxBoxPlan *out) {
  FluxPlan f{d, *out};
  return flux_select(d, dir, f);
}

unsigned weno_batch_blocks(const Dev &d, int dir) {
  // as the single-box launch: enough 64-thread CTAs for every slot, at
  // most 16 per multiprocessor (the list length is known on the device only)
  long long need = (d.nslot[dir] + WENO_NT - 1) / WENO_NT;
  long long cap = (long long)(d.weno_cps > 0 ? d.weno_cps : 16) * d.nsm;
  return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

cudaError_t launch_flux_batch(const Dev &d0, const BatchArgs &ba, unsigned total, const FluxMaps *maps,
                              const void *tgs, int dir, int accumulate, cudaStream_t st) {
  FluxBatchLaunch f{ba, total, maps, tgs, accumulate, st};
  return flux_select(d0, dir, f);
}

cudaError_t launch_weno_batch(const Dev &d0, const BatchArgs &ba, unsigned total, int dir, cudaStream_t st) {
  return d0.mixed ? weno_batch_dir<float>(d0, ba, total, dir, st) : weno_batch_dir<double>(d0, ba, total, dir, st);
}

}  // namespace s2
