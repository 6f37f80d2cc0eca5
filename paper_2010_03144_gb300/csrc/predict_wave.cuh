// K2 for large cube blocks (B = 12, 16): the prediction loop of Algorithm 1 with the rows of
// a block spread over the lanes of a warp and an anti-diagonal wavefront inside the block.
//
// Why: the one-thread-per-block walk keeps a B x B plane of reconstructed values per thread
// (1 KB at 16^3 float32), so only a few warps fit on an SM and each walks 4096 points in
// sequence. Here lane j of a block owns the block's rows (i, j, *) for every plane i, and lane
// j runs one step behind lane j - 1: at step t it handles point (i, j, l) with
// i * B + l = t - j. Every Lorenzo neighbour is then ready when it is needed:
//   (i, j, l-1)     this lane, step t-1          (i-1, j, l)     this lane, step t-B
//   (i, j-1, l)     lane j-1, step t-1           (i-1, j-1, l)   read by lane j-1 at step t-1
//   (i, j-1, l-1)   lane j-1, step t-2           (i-1, j, l-1), (i-1, j-1, l-1): one step earlier
// so a point is predicted from the same reconstructed values, with the same operations in the
// same order, as in the sequential walk: codes, reconstructed values and checksums are the
// sequential ones bit for bit (the checksums are integer sums, so their order is free). The
// previous plane's values stay in registers: lane j keeps x'(i-1, j, l) in slot (l + j) mod B
// of a B-register array, which step t reads and overwrites at the compile-time index t mod B.
//
// A CTA takes G consecutive blocks at a time (a lane group of B lanes per block, 32 / B blocks
// per warp). The input reaches shared memory plane by plane through a ring of three plane
// slots filled by cp.async one plane ahead; codes go to a ring of three plane slots in shared
// memory and are written out plane by plane in the warp-interleaved pair layout (G blocks'
// pairs are G consecutive words: whole 32-byte sectors). One barrier per plane.
//
// Per block, as in the one-thread walk: the predictor choice (E_reg over the sample rows, each
// lane summing the terms of one row, the sum itself taken in the sequential order), the
// unvoted duplicate checks collected in a mask, and at the end the checks of Algorithm 1. A
// block whose duplicate evaluations disagreed, which carries soft-error records, or whose input
// checksums do not match is walked again by its first lane with the voting walk of the generic
// path (the same values; the re-walk and the repair are counted as there).
#pragma once

namespace sdcsz {
namespace kpred {
namespace {

template <typename T, int B, int G>
struct WaveCfg {
  static constexpr int BPW = 32 / B;                      // blocks per warp
  static constexpr int NW = (G + BPW - 1) / BPW;          // warps per CTA
  static constexpr int NT = 32 * NW;
  static constexpr int MINB = NW >= 16 ? 1 : 16 / NW;    // CTAs per SM the registers are sized for
  static constexpr int ES = (int)sizeof(T);
  static constexpr int RP = B + ((16 - (B * ES) % 16) % 16) / ES;  // input row pitch (elements)
  static constexpr int PLANE = G * B * RP;                // elements per input ring slot
  static constexpr int CPL = B * B + 4;                   // halfwords per block plane in the code ring
  static constexpr int WSLOTS = B * B + B;                // generic walk slots (walker_slots)
  static constexpr size_t RING = (size_t)3 * PLANE * ES;
  static constexpr size_t SCRATCH = (size_t)G * WSLOTS * ES;
  static constexpr size_t CODES = (size_t)3 * G * CPL * 2;
  static constexpr size_t SMEM = (RING > SCRATCH ? RING : SCRATCH) + CODES;
  static_assert(B % 2 == 0, "pairs of codes never straddle a row");
  static_assert(32 % G == 0, "a group stays inside one interleave group of 32 blocks");
};

// Row j of block q in the input ring: the two blocks of a 16-lane warp half interleave their
// rows (j ^ 1 for odd q), which keeps the skewed reads of a warp on distinct banks.
template <int B>
__device__ __forceinline__ int ring_row(int q, int j) {
  return B == 16 ? (j ^ (q & 1)) : j;
}

__device__ __forceinline__ void cp_async_sz(void* dst_smem, const void* src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_w() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One thread per block row (thread t < G * B: block t / B, row t % B): the row's source in the
// field (plane 0), its place in a ring slot, its length and the block's planes, set once per
// group. Edge blocks copy element by element (their rows need not start on a wider boundary).
struct FillRow {
  const char* src;  // nullptr: no row (no block, or a row past the block's extent)
  uint32_t dst;     // byte offset in ring slot 0
  int nbytes, cb;   // row bytes, copy size
  int planes;       // planes of the block
};

template <typename T, int B, int G>
__device__ __forceinline__ FillRow fill_row(const T* __restrict__ field, const uint64_t* s_base, const uint32_t* s_ext,
                                            uint64_t sj, int cb) {
  typedef WaveCfg<T, B, G> C;
  FillRow f;
  f.src = nullptr;
  f.dst = 0;
  f.nbytes = 0;
  f.cb = cb;
  f.planes = 0;
  const int t = threadIdx.x;
  if (t < G * B) {
    const int q = t / B, j = t - (t / B) * B;
    const uint64_t base = s_base[q];
    const uint32_t ex = s_ext[q];
    const int e0 = ex & 255, e1 = (ex >> 8) & 255, e2 = ex >> 16;
    if (base != ~0ull && j < e1) {
      f.src = reinterpret_cast<const char*>(field + base + (uint64_t)j * sj);
      f.dst = (uint32_t)((q * B + ring_row<B>(q, j)) * C::RP * C::ES);
      f.nbytes = e2 * C::ES;
      f.planes = e0;
      if (e0 != B || e1 != B || e2 != B) f.cb = C::ES;
    }
  }
  return f;
}

// Plane pl of this thread's row into ring slot `slot`.
template <typename T, int B, int G>
__device__ __forceinline__ void wave_fill(unsigned char* ring, int slot, int pl, const FillRow& f, uint64_t si_bytes) {
  typedef WaveCfg<T, B, G> C;
  if (!f.src || pl >= f.planes) return;
  const char* src = f.src + (uint64_t)pl * si_bytes;
  unsigned char* dst = ring + (size_t)slot * C::PLANE * C::ES + f.dst;
  for (int o = 0; o < f.nbytes; o += f.cb) cp_async_sz(dst + o, src + o, f.cb);
}

// The codes of plane pl (code ring slot pl % 3) to the interleaved pair layout. Groups of full
// blocks: word p of block q goes to pair line p, lane (b0 & 31) + q, G blocks' words side by
// side. Groups of edge blocks (extents e0 x e1 x e2): code by code at their block-local index.
// Thread t always serves block t % G.
template <typename T, int B, int G>
__device__ __forceinline__ void wave_flush(const uint16_t* cring, int pl, const Geo& g, const Ws& w, uint64_t b0,
                                           uint64_t bq, uint32_t extq, bool edge) {
  typedef WaveCfg<T, B, G> C;
  constexpr int PP = B * B / 2;  // pairs per block plane
  if (bq == ~0ull) return;
  const int q = threadIdx.x % G;
  if (!edge) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(cring) + (size_t)((pl % 3) * G + q) * (C::CPL / 2);
    uint32_t* dst = reinterpret_cast<uint32_t*>(w.codes) +
                    ((b0 >> 5) * (uint64_t)pairs_of(g.P) + (uint64_t)pl * PP) * 32 + (b0 & 31) + q;
#pragma unroll 4
    for (int p = threadIdx.x / G; p < PP; p += C::NT / G) dst[(uint64_t)p * 32] = src[p];
    return;
  }
  const int e0 = extq & 255, e1 = (extq >> 8) & 255, e2 = extq >> 16;
  if (pl >= e0) return;
  const uint16_t* src = cring + (size_t)((pl % 3) * G + q) * C::CPL;
  const uint32_t k0 = (uint32_t)(pl * e1 * e2);
  for (int idx = threadIdx.x / G; idx < e1 * e2; idx += C::NT / G) {
    const int jj = idx / e2, ll = idx - jj * e2;
    w.codes[code_pos(bq, g.P, k0 + idx)] = src[jj * B + ll];
  }
}

// Segmented sum over the B lanes of a block (the result in its lane j = 0).
template <int B, typename V>
__device__ __forceinline__ V seg_sum(V v, int j) {
#pragma unroll
  for (int o = 1; o < B; o <<= 1) {
    const V u = __shfl_down_sync(0xffffffffu, v, o);
    if (j + o < B) v += u;
  }
  return v;
}
template <int B>
__device__ __forceinline__ uint32_t seg_or(uint32_t v, int j) {
#pragma unroll
  for (int o = 1; o < B; o <<= 1) {
    const uint32_t u = __shfl_down_sync(0xffffffffu, v, o);
    if (j + o < B) v |= u;
  }
  return v;
}

// The predictor of the blocks a warp holds, the same for all of them or not: Lorenzo only,
// regression only, or both evaluated and one chosen per lane (warp-uniform, so that every
// shuffle of a step is taken by the whole warp).
constexpr int kModeLor = 0, kModeReg = 1, kModeMix = 2;

// One group of G blocks (all the CTA's threads): full blocks b0 .. b0 + G - 1 of the field (cut
// ones skipped), or, with `edge`, entries b0 .. b0 + G - 1 of the compact enumeration of the cut
// blocks, each with its own extents. `count` bounds the block (or entry) indices.
template <typename T, int B, int G, bool ABFT, bool CMP>
__device__ __forceinline__ void wave_group(const T* __restrict__ field, const Geo& g, const Ws& w,
                                           const sdcsz_flip* __restrict__ flips, uint32_t nflips, bool edge,
                                           uint64_t grp, uint64_t count, unsigned char* smem, uint64_t* s_base,
                                           uint32_t* s_ext, uint64_t* s_blk, const Hist& h, const Consts<T>& K,
                                           Counters& cnt) {
  typedef WaveCfg<T, B, G> C;
  constexpr uint32_t P = B * B * B;
  constexpr unsigned FULL = 0xffffffffu;
  T* ring = reinterpret_cast<T*>(smem);
  uint16_t* cring = reinterpret_cast<uint16_t*>(smem + (C::RING > C::SCRATCH ? C::RING : C::SCRATCH));
  T* ustage = static_cast<T*>(w.ustage);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qw = lane / B, j = lane - qw * B;
  const int q = warp * C::BPW + qw;
  const bool lane_used = qw < C::BPW && q < G;
  const int qs = lane_used ? q : 0;  // ring index (lanes without a block read block 0's rows)
  const uint64_t si = g.d[1] * g.d[2], sj = g.d[2];
  const int lbase = lane - j;  // lane of this block's row 0
  const uint32_t R = g.R;
  const int rrow = (qs * B + ring_row<B>(qs, j)) * C::RP;  // this lane's row in a ring slot
  const int crow = qs * C::CPL + j * B;                     // and in a code ring slot
  // the widest copy every row start of every full block allows, and two-value row loads
  const uintptr_t fp = reinterpret_cast<uintptr_t>(field);
  int cb = C::ES;
  if ((B * C::ES) % 16 == 0 && (g.d[2] * C::ES) % 16 == 0 && fp % 16 == 0) cb = 16;
  else if (C::ES < 8 && (B * C::ES) % 8 == 0 && (g.d[2] * C::ES) % 8 == 0 && fp % 8 == 0) cb = 8;
  const bool vec2 = (g.d[2] % 2 == 0) && (fp % (2 * C::ES) == 0);
  uint32_t run_n = 0;  // central codes counted in a register (added to the histogram at the end)
  // this lane's block: a full block of the field (blocks b0 .. b0 + G - 1, cut ones skipped),
  // or an edge block (the compact enumeration of the cut ones) with its own extents
  const uint64_t b0 = grp * G, e = b0 + q;
  bool full = false;  // "the block is walked here"
  uint64_t b = 0, base = ~0ull;
  int e0 = B, e1 = B, e2 = B;
  if (lane_used && e < count) {
    uint64_t c0, c1, c2;
    b = edge ? edge_block(g, e) : e;
    block_coords(g, b, c0, c1, c2);
    if (edge) {
      e0 = (int)min((uint64_t)B, g.d[0] - c0 * B);
      e1 = (int)min((uint64_t)B, g.d[1] - c1 * B);
      e2 = (int)min((uint64_t)B, g.d[2] - c2 * B);
      full = true;
    } else {
      full = (c0 + 1) * B <= g.d[0] && (c1 + 1) * B <= g.d[1] && (c2 + 1) * B <= g.d[2];
    }
    if (full) base = (c0 * B * g.d[1] + c1 * B) * g.d[2] + c2 * B;
  }
  if (lane_used && j == 0) {
    s_base[q] = base;
    s_ext[q] = (uint32_t)e0 | ((uint32_t)e1 << 8) | ((uint32_t)e2 << 16);
    s_blk[q] = b;
  }
  __syncthreads();
  const FillRow fr = fill_row<T, B, G>(field, s_base, s_ext, sj, cb);
  const uint64_t bq = s_base[threadIdx.x % G] != ~0ull ? s_blk[threadIdx.x % G] : ~0ull;  // flush's block
  const uint32_t extq = s_ext[threadIdx.x % G];
  wave_fill<T, B, G>(smem, 0, 0, fr, si * C::ES);
  cp_async_commit_w();

  // predictor choice: E_reg over the sample rows (i, i); lane j sums the terms of row j and
  // the rows are added in order
  CoefSel cq;
  cq.c4 = make_float4(0.f, 0.f, 0.f, 0.f);
  cq.ok = false;
  float terms[B];
#pragma unroll
  for (int l = 0; l < B; ++l) terms[l] = 0.0f;
  if (full && !edge) {
    cq = coef_select<T, 3>(g, w, b);
    T x[B];
    load_row<T, B>(field + base + (uint64_t)j * si + (uint64_t)j * sj, vec2 != 0, x);
    const float ra = __fadd_rn(__fmul_rn(cq.c4.x, (float)j), __fmul_rn(cq.c4.y, (float)j));
#pragma unroll
    for (int l = 0; l < B; ++l) {
      const float f = __fadd_rn(__fadd_rn(ra, __fmul_rn(cq.c4.z, (float)l)), cq.c4.w);
      terms[l] = fabsf(__fsub_rn(FT<T>::tofloat(x[l]), f));
    }
  }
  float E = 0.0f;
#pragma unroll 1
  for (int r = 0; r < B; ++r) {
    if (j == r) {
#pragma unroll
      for (int l = 0; l < B; ++l) E = __fadd_rn(E, terms[l]);
    }
    E = __shfl_sync(FULL, E, (lbase + r) & 31);
  }
  Box xb;  // an edge block's box
  if (edge && full) {
    cq = coef_select<T, 3>(g, w, b);
    xb = block_box(g, b);
    if (j == 0) E = ereg_generic<T, 3>(field, g, xb, cq.c4, kNone, T(0));
  }
  if (edge) E = __shfl_sync(FULL, E, lbase & 31);
  const uint32_t S = edge ? (full ? sample_points(3, xb.e) : 0u) : (uint32_t)(B * B);
  bool reg = false;
  T cT[4] = {T(0), T(0), T(0), T(0)};
  Hooks hk;
  hk.kp = hk.kr = hk.kfix = kNone;
  hk.bitp = hk.bitr = 0;
  hk.rewalk = false;
  hk.texp = K.texp;
  if (full) {
    reg = choose_reg(g, w, b, cq.ok, S, K.noise, [&] { return E; });
    load_coefs<T, 3>(g, w, b, flips, nflips, cT, hk, cq, K);
  }
  const bool any_reg = __any_sync(FULL, full && reg), any_lor = __any_sync(FULL, full && !reg);
  const int mode = any_reg ? (any_lor ? kModeMix : kModeReg) : kModeLor;

  // the wavefront: B + 1 macro-steps of B steps; in macro-step m a lane is on plane m - 1
  // for its first j steps (l = s - j + B) and on plane m after them (l = s - j)
  PassRes r = {0, 0, 0, 0, 0, 0, 0, 0};
  T prev[B];
#pragma unroll
  for (int s2 = 0; s2 < B; ++s2) prev[s2] = T(0);
  T cur_l = T(0), a_l = T(0), b_l = T(0), ab_l = T(0);
  const uint64_t cbase = code_index(b, P, 0);
  const T tj = (T)(uint32_t)j;
#pragma unroll 1
  for (int m = 0; m <= B; ++m) {
    cp_async_wait_all();
    __syncthreads();
    if (m + 1 < B) wave_fill<T, B, G>(smem, (m + 1) % 3, m + 1, fr, si * C::ES);
    cp_async_commit_w();
    if (m >= 2) wave_flush<T, B, G>(cring, m - 2, g, w, b0, bq, extq, edge != 0);
    // per lane and plane (p: plane m - 1, c: plane m)
    const int sp = (m + 2) % 3, sc = m % 3;
    const int offp = sp * C::PLANE + rrow + B - j, offc = sc * C::PLANE + rrow - j;
    const int coffp = sp * G * C::CPL + crow + B - j, coffc = sc * G * C::CPL + crow - j;
    // k = (i * e1 + j) * e2 + l; a point is in the block when i < e0, j < e1 and l < e2
    const uint32_t kp = (uint32_t)(((m - 1) * e1 + j) * e2 + B - j), kc = (uint32_t)((m * e1 + j) * e2 - j);
    const bool vp = full && j < e1 && m >= 1 && m - 1 < e0, vc = full && j < e1 && m < e0;
    const int thp = e2 + j - B, thc = e2 + j;  // l < e2 as a bound on s
    const bool ap = m >= 2, ac0 = m >= 1;
    T rp = T(0), rc = T(0), rpv = T(0), rcv = T(0);  // regression: c0 * i + c1 * j, both evaluations
    if (mode != kModeLor) {
      const T ti_p = (T)(uint32_t)max(m - 1, 0), ti_c = (T)(uint32_t)m;
      rp = FT<T>::add(FT<T>::mul(cT[0], ti_p), FT<T>::mul(cT[1], tj));
      rc = FT<T>::add(FT<T>::mul(cT[0], ti_c), FT<T>::mul(cT[1], tj));
      rpv = FT<T>::add_v(FT<T>::mul_v(cT[0], ti_p), FT<T>::mul_v(cT[1], tj));
      rcv = FT<T>::add_v(FT<T>::mul_v(cT[0], ti_c), FT<T>::mul_v(cT[1], tj));
    }
    auto steps = [&](auto md) {
      constexpr int MODE = decltype(md)::value;
#pragma unroll
      for (int s = 0; s < B; ++s) {
        const bool wr = s < j;  // still on plane m - 1
        const bool valid = (wr ? vp : vc) && s < (wr ? thp : thc);
        const T v = ring[(wr ? offp : offc) + s];
        T bn = T(0), abn = T(0), a = T(0);
        T c = T(0), ac = T(0), bc = T(0), abc = T(0);
        if (MODE != kModeReg) {
          bn = __shfl_up_sync(FULL, cur_l, 1);
          abn = __shfl_up_sync(FULL, a_l, 1);
          if (j == 0) {
            bn = T(0);
            abn = T(0);
          }
          if (s != j) {  // l > 0
            c = cur_l;
            ac = a_l;
            bc = b_l;
            abc = ab_l;
          }
          if (wr ? ap : ac0) a = prev[s];
        }
        uint32_t mm1 = 0, dup0 = 0;
        T pred;
        if (MODE == kModeLor) {
          pred = dup_pred<T, ABFT, false>([&] { return lorenzo_of<T, 3, OpRN<T>>(a, bn, abn, ac, bc, abc, c); },
                                          [&] { return lorenzo_of<T, 3, OpV<T>>(a, bn, abn, ac, bc, abc, c); },
                                          false, 0u, dup0, mm1);
        } else {
          const T tl = (T)(uint32_t)(wr ? s - j + B : s - j);
          const T ra = wr ? rp : rc, rv = wr ? rpv : rcv;
          const T pr = dup_pred<T, ABFT, false>(
              [&] { return FT<T>::add(FT<T>::add(ra, FT<T>::mul(cT[2], tl)), cT[3]); },
              [&] { return FT<T>::add_v(FT<T>::add_v(rv, FT<T>::mul_v(cT[2], tl)), cT[3]); }, false, 0u, dup0,
              mm1);
          if (MODE == kModeReg) {
            pred = pr;
          } else {
            const T pl = dup_pred<T, ABFT, false>(
                [&] { return lorenzo_of<T, 3, OpRN<T>>(a, bn, abn, ac, bc, abc, c); },
                [&] { return lorenzo_of<T, 3, OpV<T>>(a, bn, abn, ac, bc, abc, c); }, false, 0u, dup0, mm1);
            pred = reg ? pr : pl;
          }
        }
        T xr;
        const uint32_t code = quantize<T, ABFT, false, CMP>(v, pred, K.eb, K.inv2, K.Rh, R, false, 0u, xr, dup0,
                                                            mm1, hk.texp);
        if (valid) cring[(wr ? coffp : coffc) + s] = (uint16_t)code;
        const uint32_t k = (wr ? kp : kc) + (uint32_t)s;
        const uint32_t vm = valid ? 0xffffffffu : 0u;
        run_n += (valid && code == R) ? 1u : 0u;
        if (valid && code != R) {
          h.add(code, 1u);
          if (!code) {
            ustage[cbase + (uint64_t)k * 32] = v;
            ++r.nun;
          }
        }
        if (ABFT) {
          r.mm |= mm1 & vm;
          const uint32_t w0 = FT<T>::lo(v) & vm;
          if (FT<T>::W == 1) {
            mad_wide(r.sw, w0, 1u);
            mad_wide(r.isw, w0, k + 1);
          } else {
            const uint32_t w1 = FT<T>::hi(v) & vm;
            mad_wide(r.sw, w0, 1u);
            mad_wide(r.sw, w1, 1u);
            mad_wide(r.isw, w0, 2 * k + 1);
            mad_wide(r.isw, w1, 2 * k + 2);
          }
          const uint32_t cm = code & vm;
          r.sq += cm;
          mad_wide(r.isq, cm, k + 1);
          mad_wide(r.sdc, FT<T>::lo(xr) & vm, 1u);
          if (FT<T>::W == 2) mad_wide(r.sdc, FT<T>::hi(xr) & vm, 1u);
        }
        if (MODE != kModeReg) {
          prev[s] = xr;
          cur_l = xr;
          a_l = a;
          b_l = bn;
          ab_l = abn;
        }
      }
    };
    if (mode == kModeLor) steps(std::integral_constant<int, kModeLor>());
    else if (mode == kModeReg) steps(std::integral_constant<int, kModeReg>());
    else steps(std::integral_constant<int, kModeMix>());
  }
  __syncthreads();
  wave_flush<T, B, G>(cring, B - 1, g, w, b0, bq, extq, edge != 0);
  // the block's sums in its row-0 lane
  r.sw = seg_sum<B>(r.sw, j);
  r.isw = seg_sum<B>(r.isw, j);
  r.isq = seg_sum<B>(r.isq, j);
  r.sdc = seg_sum<B>(r.sdc, j);
  r.sq = seg_sum<B>(r.sq, j);
  r.nun = seg_sum<B>(r.nun, j);
  r.mm = seg_or<B>(r.mm, j);
  if (run_n) {
    h.add(R, run_n);
    run_n = 0;
  }
  __syncthreads();  // the codes written by the flush are visible to the re-walks below
  if (full && j == 0) {
    Walker<T, 3> wk;
    wk.base = ring + (size_t)q * C::WSLOTS;
    wk.stride = 1;
    wk.B2 = B;
    wk.sr = B * B;
    const Box x = block_box(g, b);
    const uint32_t Pb = x.P;
    const bool hooked = (hk.kp != kNone) || (hk.kr != kNone);
    if (ABFT && (hooked || r.mm || hk.rewalk)) {
      // voting walk: the block's codes leave the histogram and come back with the walk
      withdraw(w, g, b, Pb, h);
      r = reg ? generic_pass<T, 3, true, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage, h, hk,
                                               T(0))
              : generic_pass<T, 3, false, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage, h, hk,
                                                T(0));
      if (!hooked) r.dup = r.dup ? r.dup : 1u;
    }
    uint8_t flag = 0;
    if (ABFT && (r.sw != w.sum_in[b] || r.isw != w.isum_in[b])) {
      uint32_t kf;
      T xf;
      if (locate_input<T>(field, g, x, w.sum_in[b], w.isum_in[b], r, &kf, &xf)) {
        withdraw(w, g, b, Pb, h);
        hk.kfix = kf;
        const CoefSel cq2 = coef_select<T, 3>(g, w, b);
        reg = choose_reg(g, w, b, cq2.ok, sample_points(3, x.e), K.noise,
                         [&] { return ereg_generic<T, 3>(field, g, x, cq2.c4, kf, xf); });
        r = reg ? generic_pass<T, 3, true, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage, h,
                                                 hk, xf)
                : generic_pass<T, 3, false, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage, h,
                                                  hk, xf);
        ++cnt.fix;
      } else {
        ++cnt.bad;
        flag = 2;
      }
    }
    block_epilogue<T>(w, b, reg, 3, cT, r, ABFT, flag, g);
    cnt.unpred += r.nun;
    cnt.reg += reg;
    cnt.dup += r.dup;
  }
  __syncthreads();  // the ring (and the re-walks' scratch in it) is free for the next group
}

template <typename T, int B, int G, bool ABFT, bool CMP>
__global__ void __launch_bounds__(WaveCfg<T, B, G>::NT, WaveCfg<T, B, G>::MINB)
    k_predict_wave(const T* __restrict__ field, Geo g, Ws w, const sdcsz_flip* __restrict__ flips, uint32_t nflips,
                   int edge, uint64_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  __shared__ uint64_t s_base[G];  // element offset of each block's origin, ~0: no block here
  __shared__ uint32_t s_ext[G];   // extents e0 | e1 << 8 | e2 << 16
  __shared__ uint64_t s_blk[G];   // block index
  State* st = w.st;
  if (*(volatile unsigned int*)&st->error) return;
  Hist h;
  hist_init(hist_s, h, g, w);
  __syncthreads();
  const Consts<T> K(st->eb, g, 3);
  Counters cnt;
  unsigned long long* queue = &st->queue[edge ? 1 : 0];
  for (uint64_t grp = cta_pull(queue); grp * G < count; grp = cta_pull(queue))
    wave_group<T, B, G, ABFT, CMP>(field, g, w, flips, nflips, edge != 0, grp, count, smem, s_base, s_ext, s_blk, h,
                                   K, cnt);
  cnt.commit(st);
  hist_flush(hist_s, h, w);
}

// Batched: every job of one block shape; a job's items are its groups of full blocks, then its
// groups of edge blocks.
template <typename T, int B, int G, bool ABFT, bool CMP>
__global__ void __launch_bounds__(WaveCfg<T, B, G>::NT, WaveCfg<T, B, G>::MINB) k_predict_wave_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  __shared__ uint64_t s_base[G];
  __shared__ uint32_t s_ext[G];
  __shared__ uint64_t s_blk[G];
  __shared__ Job s_job;
  Hist h;
  Counters cnt;
  batch_loop(
      a, s_job,
      [&] {
        hist_init(hist_s, h, s_job.g, s_job.w);
        __syncthreads();
      },
      [&](uint64_t it) {
        const Geo g = s_job.g;
        const uint64_t nfull = (g.nb + G - 1) / G;
        const bool edge = it >= nfull;
        const Consts<T> K(s_job.w.st->eb, g, 3);
        wave_group<T, B, G, ABFT, CMP>(static_cast<const T*>(s_job.field), g, s_job.w, nullptr, 0, edge,
                                       edge ? it - nfull : it, edge ? edge_count(g) : g.nb, smem, s_base, s_ext,
                                       s_blk, h, K, cnt);
      },
      [&] {
        cnt.commit(s_job.w.st);
        cnt = Counters();
        hist_flush(hist_s, h, s_job.w);
      });
}

}  // namespace
}  // namespace kpred
}  // namespace sdcsz
