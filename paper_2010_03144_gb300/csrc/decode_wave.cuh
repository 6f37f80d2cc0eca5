// K5 for large cube blocks (B = 10, 12, 16): the decompression loop of Algorithm 2 in two
// passes over the blocks, then Algorithm 2's re-execution of the blocks that failed their check.
//
//   A (one thread per block, every block at once): the block's Huffman codes, unpredictable
//     values and coefficients into the workspace, the codes in the compression's interleaved
//     pair layout; the decode's validity per block.
//   B (the wavefront of the prediction kernel: rows on lanes, one step of skew per row, the
//     previous plane in rotated registers, G blocks per CTA): each point reconstructed from its
//     code and the reconstructed values before it, in the sequential order of operations, the
//     block's sum_dc taken on the way; the values leave through a shared-memory ring of planes
//     as whole rows. A block whose decode failed or whose sum differs from the stored sum_dc is
//     listed for re-execution.
//   C (a few CTAs): each listed block decompressed again from its bytes by the generic decoder,
//     and reported corrected or uncorrectable as by the one-pass kernels.
//
// Why two passes: a block's codes come out of one serial bit stream, which one thread decodes
// at its own pace; the reconstruction needs a warp per block to keep enough points in flight.
// Between them the codes cost a write and a read of 2 bytes per point.
#pragma once

namespace sdcsz {
namespace kdec {
namespace {

// Workspace of the two passes (wave_decode_ws_bytes).
struct DWs {
  uint32_t* codes;          // code pairs, interleaved as in compression (stride P of a full block)
  void* un;                 // unpredictable values at code_index(b, P, k)
  void* coef;               // four coefficients per block (dtype)
  uint8_t* flag;            // per block: kFlagOk | kFlagReg | kFlagUnplaced | kFlagRange
  unsigned long long* fix;  // blocks to decompress again (their count in State::queue[3])
};
constexpr uint8_t kFlagOk = 1, kFlagReg = 2, kFlagUnplaced = 4, kFlagRange = 8;

inline DWs bind_dws(uint8_t* p, const Geo& g) {
  DWs d;
  d.codes = reinterpret_cast<uint32_t*>(p);
  p += wave_dws_part(g, 0);
  d.un = p;
  p += wave_dws_part(g, 1);
  d.coef = p;
  p += wave_dws_part(g, 2);
  d.flag = p;
  p += wave_dws_part(g, 3);
  d.fix = reinterpret_cast<unsigned long long*>(p);
  return d;
}
__device__ __forceinline__ uint64_t bits_used_d(const FastReader& br) { return br.used(); }
__device__ __forceinline__ uint64_t bits_used_d(const BitReader& br) { return br.used; }

// Pass A for block b (extents e0 x e1 x e2): codes, unpredictable values and coefficients;
// returns whether the block decodes (valid symbols, its unpredictable count, within its bytes).
// FAST: the unchecked reader, with a row of central codes taken in one comparison.
template <typename T, int B, bool CMP, bool FAST, class Reader>
__device__ __forceinline__ bool wave_codes_block(Reader& br, const uint8_t* __restrict__ s, const Hdr& h,
                                                 const BlockIn& bi, const Tables& tb, uint64_t b, uint32_t e0,
                                                 uint32_t e1, uint32_t e2, const DWs& dw) {
  constexpr uint32_t P = B * B * B;
  const uint32_t R = h.g.R;
  const bool reg = bi.reg_idx >= 0;
  bool ok = true;
  if (reg) {
    T cT[4] = {T(0), T(0), T(0), T(0)};
    ok = block_coefs<T, 3>(s, h, bi.reg_idx, br, cT, CMP);
    T* c = static_cast<T*>(dw.coef) + 4 * b;
#pragma unroll
    for (int a = 0; a < 4; ++a) c[a] = cT[a];
  }
  const T* un = reinterpret_cast<const T*>(s + h.L.unpred) + bi.un_off;
  T* wun = static_cast<T*>(dw.un);
  const bool full = e0 == B && e1 == B && e2 == B;
  uint32_t rbits = tb.rbits, rpat = tb.rpat;
  if (FAST && rbits && e2 != B) {  // a central row of an edge block: e2 central codewords
    const uint32_t lc = rbits / B;
    rbits = lc * e2;
    rpat >>= lc * (B - e2);
  }
  uint32_t used_u = 0, k = 0, lowc = 0;
  auto emit = [&](uint32_t code) {  // code k of the block
    if (full) {
      if (k & 1) dw.codes[pair_index(b, P, k)] = lowc | (code << 16);
      else lowc = code;
    } else {
      reinterpret_cast<uint16_t*>(dw.codes)[code_pos(b, P, k)] = (uint16_t)code;
    }
    ++k;
  };
  for (uint32_t i = 0; i < e0; ++i) {
    for (uint32_t j = 0; j < e1; ++j) {
      if constexpr (FAST) {
        if (ok && rbits && (br.peek() >> (32 - rbits)) == rpat) {
          br.advance(rbits);
          for (uint32_t l = 0; l < e2; ++l) emit(R);
          continue;
        }
      }
      int qp = kDefer;  // the second symbol of a pair decoded with the previous one
      for (uint32_t l = 0; l < e2; ++l) {
        int q;
        if constexpr (FAST) {
          // rows of even length: symbols in pairs from one lookup where both fit the window
          if (!ok) {
            q = -1;
          } else if (!(e2 & 1) && !(l & 1)) {
            br.next2(tb.lut2, tb.lut, *tb.cn, tb.syms, tb.n_live, q, qp, CMP);
          } else if (!(e2 & 1)) {
            q = (qp == kDefer) ? br.next(tb.lut, *tb.cn, tb.syms, tb.n_live) : qp;
          } else {
            q = br.next(tb.lut, *tb.cn, tb.syms, tb.n_live);
          }
        } else {
          q = ok ? br.next(tb.lut, *tb.cn, tb.syms, tb.n_live) : -1;
        }
        uint32_t code = 0;
        if (q < 0 || (uint32_t)q >= h.g.bins) {
          ok = false;
        } else if (q == 0) {
          if (used_u >= bi.ucnt) {
            ok = false;
          } else {
            const T v = CMP ? read_unpred<T>(br, h.texp) : un[used_u];
            wun[code_index(b, P, k)] = v;
          }
          ++used_u;
        } else {
          code = (uint32_t)q;
        }
        emit(code);
      }
    }
  }
  if (used_u != bi.ucnt || bits_used_d(br) > (uint64_t)bi.size * 8u) ok = false;
  return ok;
}

// Pass A: warp items of 32 consecutive blocks (placed as by the one-pass kernel), one per lane.
template <typename T, int B, bool CMP>
__global__ void __launch_bounds__(256) k_wave_codes(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h, State* st,
                                                    DWs dw) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Smem sm;
  Tables tb;
  if (!fast_tables<B, CMP>(s, h, sm, smem, st, &tb)) return;
  const uint8_t* lim = s + nbytes;
  const Geo& g = h.g;
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup, nitems = (g.nb + 31) / 32;
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t item = warp_pull(&st->queue[0]); item < nitems; item = warp_pull(&st->queue[0])) {
    BlockIn bi;
    const bool placed = warp_place(s, h, item, ngroups, st, &bi);
    const uint64_t b = 32 * item + lane;
    if (b >= g.nb) continue;
    uint8_t fl = kFlagUnplaced;
    if (placed) {
      const bool reg = bi.reg_idx >= 0;
      const bool in_range = !(bi.pay_off + bi.size > h.payload_bytes || bi.un_off + bi.ucnt > h.n_unpred ||
                              (reg && (uint64_t)bi.reg_idx >= h.n_reg));
      fl = kFlagRange;
      if (in_range) {
        uint64_t c0, c1, c2;
        block_coords(g, b, c0, c1, c2);
        const uint32_t e0 = (uint32_t)min((uint64_t)B, g.d[0] - c0 * B);
        const uint32_t e1 = (uint32_t)min((uint64_t)B, g.d[1] - c1 * B);
        const uint32_t e2 = (uint32_t)min((uint64_t)B, g.d[2] - c2 * B);
        // the unchecked reader's reach (as in the one-pass kernel), else the checked one
        const uint64_t worst = CMP ? (3ull + sizeof(T)) * (B * B * B) + 19 : 3ull * (B * B * B);
        const bool safe = (uint64_t)(lim - (s + h.L.payload)) >= bi.pay_off + worst + 16;
        {  // the block's payload on its way to L2 (the reader then waits on L2, not on DRAM)
          const uint64_t p0 = h.L.payload + bi.pay_off, p1 = min(p0 + bi.size, nbytes);
          for (uint64_t o = p0 & ~uint64_t(127); o < p1; o += 128) prefetch_l2(s + o);
        }
        bool ok;
        if (safe) {
          FastReader br;
          br.init(s + h.L.payload + bi.pay_off);
          ok = wave_codes_block<T, B, CMP, true>(br, s, h, bi, tb, b, e0, e1, e2, dw);
        } else {
          BitReader br;
          br.init(s + h.L.payload + bi.pay_off, lim);
          ok = wave_codes_block<T, B, CMP, false>(br, s, h, bi, tb, b, e0, e1, e2, dw);
        }
        fl = (ok ? kFlagOk : 0) | (reg ? kFlagReg : 0);
      }
    }
    dw.flag[b] = fl;
  }
}

// ---------------------------------------------------------------- pass B
template <typename T, int B, int G>
struct DWaveCfg {
  static constexpr int BPW = 32 / B;              // blocks per warp
  static constexpr int NW = (G + BPW - 1) / BPW;  // warps per CTA
  static constexpr int NT = 32 * NW;
  static constexpr int MINB = NW >= 16 ? 1 : 16 / NW;
  static constexpr int ES = (int)sizeof(T);
  static constexpr int RP = B + ((16 - (B * ES) % 16) % 16) / ES;  // output row pitch (elements)
  static constexpr int PLANE = G * B * RP;                        // elements per output ring slot
  static constexpr int CPL = B * B + 4;                           // halfwords per block plane of codes
  static constexpr size_t ORING = (size_t)3 * PLANE * ES;
  static constexpr size_t SMEM = ORING + (size_t)3 * G * CPL * 2;
  static_assert(B % 2 == 0, "pairs of codes never straddle a row");
  static_assert(32 % G == 0, "a group stays inside one interleave group of 32 blocks");
};

template <int B>
__device__ __forceinline__ int dring_row(int q, int j) {
  return B == 16 ? (j ^ (q & 1)) : j;
}
__device__ __forceinline__ void dcp_async4(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void dcp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void dcp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int B, typename V>
__device__ __forceinline__ V dseg_sum(V v, int j) {
#pragma unroll
  for (int o = 1; o < B; o <<= 1) {
    const V u = __shfl_down_sync(0xffffffffu, v, o);
    if (j + o < B) v += u;
  }
  return v;
}

// The codes of plane pl of the group's blocks into code ring slot pl % 3: full blocks by
// 4-byte copies of their pair words (G words of a pair line side by side), edge blocks code by
// code. Thread t serves block t % G.
template <typename T, int B, int G>
__device__ __forceinline__ void wave_code_fill(uint16_t* cring, int pl, const Geo& g, const DWs& dw, uint64_t b0,
                                               uint64_t bq, uint32_t extq, bool edge) {
  typedef DWaveCfg<T, B, G> C;
  constexpr int PP = B * B / 2;
  constexpr uint32_t P = B * B * B;
  if (bq == ~0ull) return;
  const int q = threadIdx.x % G;
  if (!edge) {
    uint32_t* dst = reinterpret_cast<uint32_t*>(cring) + (size_t)((pl % 3) * G + q) * (C::CPL / 2);
    const uint32_t* src = dw.codes + ((b0 >> 5) * (uint64_t)pairs_of(P) + (uint64_t)pl * PP) * 32 + (b0 & 31) + q;
    for (int p = threadIdx.x / G; p < PP; p += C::NT / G) dcp_async4(dst + p, src + (uint64_t)p * 32);
    return;
  }
  const int e0 = extq & 255, e1 = (extq >> 8) & 255, e2 = extq >> 16;
  if (pl >= e0) return;
  uint16_t* dst = cring + (size_t)((pl % 3) * G + q) * C::CPL;
  const uint16_t* src = reinterpret_cast<const uint16_t*>(dw.codes);
  const uint32_t k0 = (uint32_t)(pl * e1 * e2);
  for (int idx = threadIdx.x / G; idx < e1 * e2; idx += C::NT / G) {
    const int jj = idx / e2, ll = idx - jj * e2;
    dst[jj * B + ll] = src[code_pos(bq, P, k0 + idx)];
  }
}

// Plane pl of the group's output ring (slot pl % 3) to the field: thread t < G * B writes row
// t % B of block t / B, in 16-byte stores where every row allows them.
template <typename T, int B, int G>
__device__ __forceinline__ void wave_out_flush(const T* oring, int pl, T* __restrict__ field, const uint64_t* s_base,
                                               const uint32_t* s_ext, uint64_t si, uint64_t sj, bool vec16) {
  typedef DWaveCfg<T, B, G> C;
  const int t = threadIdx.x;
  if (t >= G * B) return;
  const int q = t / B, j = t - (t / B) * B;
  const uint64_t base = s_base[q];
  const uint32_t ex = s_ext[q];
  const int e0 = ex & 255, e1 = (ex >> 8) & 255, e2 = ex >> 16;
  if (base == ~0ull || j >= e1 || pl >= e0) return;
  const T* src = oring + (size_t)(pl % 3) * C::PLANE + (q * B + dring_row<B>(q, j)) * C::RP;
  T* dst = field + base + (uint64_t)pl * si + (uint64_t)j * sj;
  if (vec16 && e2 == B) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int o = 0; o < B * C::ES / 16; ++o) __stcs(d4 + o, s4[o]);
  } else {
    for (int l = 0; l < e2; ++l) __stcs(dst + l, src[l]);
  }
}

constexpr int kDModeLor = 0, kDModeReg = 1, kDModeMix = 2;

// The 3D Lorenzo prediction from its seven reconstructed neighbours, in the order of the one-pass
// decoder (and of compression): ((((a + b) - ab) - ac) - bc) + abc, then + c.
template <typename T>
__device__ __forceinline__ T dlorenzo(T a, T bb, T ab, T ac, T bc, T abc, T c) {
  T s = FT<T>::add(a, bb);
  s = FT<T>::sub(s, ab);
  s = FT<T>::sub(s, ac);
  s = FT<T>::sub(s, bc);
  s = FT<T>::add(s, abc);
  return FT<T>::add(s, c);
}

// Pass B: items are the groups of G full blocks of the field (cut ones skipped), then the
// groups of G edge blocks (compact enumeration).
template <typename T, int B, int G, bool CMP>
__global__ void __launch_bounds__(DWaveCfg<T, B, G>::NT, DWaveCfg<T, B, G>::MINB)
    k_wave_recon(const uint8_t* __restrict__ s, Hdr h, T* __restrict__ field, uint8_t* status, State* st, DWs dw) {
  typedef DWaveCfg<T, B, G> C;
  constexpr uint32_t P = B * B * B;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint64_t s_base[G];  // element offset of each block's origin, ~0: no block here
  __shared__ uint32_t s_ext[G];   // extents e0 | e1 << 8 | e2 << 16
  __shared__ uint64_t s_blk[G];   // block index
  T* oring = reinterpret_cast<T*>(smem);
  uint16_t* cring = reinterpret_cast<uint16_t*>(smem + C::ORING);
  if (*(volatile unsigned int*)&st->error) return;
  const Geo& g = h.g;
  const T eb = (T)h.eb;
  const int R = (int)g.R;
  const T* wun = static_cast<const T*>(dw.un);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qw = lane / B, j = lane - qw * B;
  const int q = warp * C::BPW + qw;
  const bool lane_used = qw < C::BPW && q < G;
  const int qs = lane_used ? q : 0;
  const uint64_t si = g.d[1] * g.d[2], sj = g.d[2];
  const int orow = (qs * B + dring_row<B>(qs, j)) * C::RP;  // this lane's row in an output ring slot
  const int crow = qs * C::CPL + j * B;                      // and in a code ring slot
  const uintptr_t fp = reinterpret_cast<uintptr_t>(field);
  const bool vec16 = (B * C::ES) % 16 == 0 && (g.d[2] * C::ES) % 16 == 0 && fp % 16 == 0;
  const uint64_t nfull = (g.nb + G - 1) / G, nedge = (edge_count(g) + G - 1) / G;
  unsigned long long bad = 0;
  for (uint64_t it = cta_pull(&st->queue[2]); it < nfull + nedge; it = cta_pull(&st->queue[2])) {
    const bool edge = it >= nfull;
    const uint64_t b0 = (edge ? it - nfull : it) * G, e = b0 + q, count = edge ? edge_count(g) : g.nb;
    bool walk = false;
    uint64_t b = 0, base = ~0ull;
    int e0 = B, e1 = B, e2 = B;
    uint8_t fl = 0;
    if (lane_used && e < count) {
      uint64_t c0, c1, c2;
      b = edge ? edge_block(g, e) : e;
      block_coords(g, b, c0, c1, c2);
      e0 = (int)min((uint64_t)B, g.d[0] - c0 * B);
      e1 = (int)min((uint64_t)B, g.d[1] - c1 * B);
      e2 = (int)min((uint64_t)B, g.d[2] - c2 * B);
      const bool full = e0 == B && e1 == B && e2 == B;
      fl = dw.flag[b];
      walk = (edge != full) && !(fl & (kFlagUnplaced | kFlagRange));
      if (walk) base = (c0 * B * g.d[1] + c1 * B) * g.d[2] + c2 * B;
    }
    if (lane_used && j == 0) {
      s_base[q] = base;
      s_ext[q] = (uint32_t)e0 | ((uint32_t)e1 << 8) | ((uint32_t)e2 << 16);
      s_blk[q] = b;
    }
    __syncthreads();
    const uint64_t bq = s_base[threadIdx.x % G] != ~0ull ? s_blk[threadIdx.x % G] : ~0ull;
    const uint32_t extq = s_ext[threadIdx.x % G];
    wave_code_fill<T, B, G>(cring, 0, g, dw, b0, bq, extq, edge);
    dcp_commit();
    const bool reg = walk && (fl & kFlagReg);
    T cT[4] = {T(0), T(0), T(0), T(0)};
    if (reg) {
      const T* c = static_cast<const T*>(dw.coef) + 4 * b;
#pragma unroll
      for (int a = 0; a < 4; ++a) cT[a] = c[a];
    }
    const unsigned long long ref = (walk && j == 0 && g.abft) ? ld_u64(s + h.L.sumdc + 8 * b) : 0ull;
    const bool any_reg = __any_sync(FULL, reg), any_lor = __any_sync(FULL, walk && !reg);
    const int mode = any_reg ? (any_lor ? kDModeMix : kDModeReg) : kDModeLor;
    const uint64_t ubase = code_index(b, P, 0);
    const T tj = (T)(uint32_t)j;
    unsigned long long sum = 0;
    T prev[B];
#pragma unroll
    for (int s2 = 0; s2 < B; ++s2) prev[s2] = T(0);
    T cur_l = T(0), a_l = T(0), b_l = T(0), ab_l = T(0);
#pragma unroll 1
    for (int m = 0; m <= B; ++m) {
      dcp_wait_all();
      __syncthreads();
      if (m + 1 < B) wave_code_fill<T, B, G>(cring, m + 1, g, dw, b0, bq, extq, edge);
      dcp_commit();
      if (m >= 2) wave_out_flush<T, B, G>(oring, m - 2, field, s_base, s_ext, si, sj, vec16);
      const int sp = (m + 2) % 3, sc = m % 3;
      const int ooffp = sp * C::PLANE + orow + B - j, ooffc = sc * C::PLANE + orow - j;
      const int coffp = sp * G * C::CPL + crow + B - j, coffc = sc * G * C::CPL + crow - j;
      const uint32_t kp = (uint32_t)(((m - 1) * e1 + j) * e2 + B - j), kc = (uint32_t)((m * e1 + j) * e2 - j);
      const bool vp = walk && j < e1 && m >= 1 && m - 1 < e0, vc = walk && j < e1 && m < e0;
      const int thp = e2 + j - B, thc = e2 + j;
      const bool ap = m >= 2, ac0 = m >= 1;
      T rp = T(0), rc = T(0);
      if (mode != kDModeLor) {
        rp = FT<T>::add(FT<T>::mul(cT[0], (T)(uint32_t)max(m - 1, 0)), FT<T>::mul(cT[1], tj));
        rc = FT<T>::add(FT<T>::mul(cT[0], (T)(uint32_t)m), FT<T>::mul(cT[1], tj));
      }
      auto steps = [&](auto md) {
        constexpr int MODE = decltype(md)::value;
#pragma unroll
        for (int s2 = 0; s2 < B; ++s2) {
          const bool wr = s2 < j;
          const bool valid = (wr ? vp : vc) && s2 < (wr ? thp : thc);
          const int code = (int)cring[(wr ? coffp : coffc) + s2];
          T bn = T(0), abn = T(0), a = T(0);
          T c = T(0), ac = T(0), bc = T(0), abc = T(0);
          if (MODE != kDModeReg) {
            bn = __shfl_up_sync(FULL, cur_l, 1);
            abn = __shfl_up_sync(FULL, a_l, 1);
            if (j == 0) {
              bn = T(0);
              abn = T(0);
            }
            if (s2 != j) {
              c = cur_l;
              ac = a_l;
              bc = b_l;
              abc = ab_l;
            }
            if (wr ? ap : ac0) a = prev[s2];
          }
          T pred;
          const T pl = dlorenzo<T>(a, bn, abn, ac, bc, abc, c);
          if (MODE == kDModeLor) {
            pred = pl;
          } else {
            const T tl = (T)(uint32_t)(wr ? s2 - j + B : s2 - j);
            const T pr = FT<T>::add(FT<T>::add(wr ? rp : rc, FT<T>::mul(cT[2], tl)), cT[3]);
            pred = (MODE == kDModeReg || reg) ? pr : pl;
          }
          T xr = FT<T>::add(pred, FT<T>::mul(FT<T>::fromi(2 * (code - R)), eb));
          if (valid && code == 0) xr = wun[ubase + (uint64_t)((wr ? kp : kc) + (uint32_t)s2) * 32];
          if (valid) oring[(wr ? ooffp : ooffc) + s2] = xr;
          const uint32_t vm = valid ? 0xffffffffu : 0u;
          mad_wide(sum, FT<T>::lo(xr) & vm, 1u);
          if (FT<T>::W == 2) mad_wide(sum, FT<T>::hi(xr) & vm, 1u);
          if (MODE != kDModeReg) {
            prev[s2] = xr;
            cur_l = xr;
            a_l = a;
            b_l = bn;
            ab_l = abn;
          }
        }
      };
      if (mode == kDModeLor) steps(std::integral_constant<int, kDModeLor>());
      else if (mode == kDModeReg) steps(std::integral_constant<int, kDModeReg>());
      else steps(std::integral_constant<int, kDModeMix>());
    }
    __syncthreads();
    wave_out_flush<T, B, G>(oring, B - 1, field, s_base, s_ext, si, sj, vec16);
    sum = dseg_sum<B>(sum, j);
    // Algorithm 2's check of the block (as the one-pass kernels: a failed first decode or a
    // sum_dc mismatch sends the block to re-execution)
    if (lane_used && j == 0 && e < count && (edge || (e0 == B && e1 == B && e2 == B))) {
      uint8_t stv = SDCSZ_BLOCK_OK;
      bool later = false;
      if (fl & kFlagUnplaced) {
        stv = SDCSZ_BLOCK_BAD;
      } else if (fl & kFlagRange) {
        stv = SDCSZ_BLOCK_BAD;
        ++bad;
      } else if (g.abft) {
        later = !(fl & kFlagOk) || sum != ref;
      } else if (!(fl & kFlagOk)) {
        stv = SDCSZ_BLOCK_BAD;
        ++bad;
      }
      if (later) dw.fix[atomicAdd(&st->queue[3], 1ull)] = b;
      else if (status) status[b] = stv;
    }
    __syncthreads();  // the rings are free for the next group
  }
  bad = warp_sum(bad);
  if (lane == 0 && bad) atomicAdd(&st->uncorrectable, bad);
}

// Pass C: the listed blocks decompressed again from their bytes (Algorithm 2's re-execution).
template <typename T>
__global__ void __launch_bounds__(64) k_wave_fixup(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h, T* field,
                                                   uint8_t* status, State* st, DWs dw) {
  const uint64_t count = *(volatile unsigned long long*)&st->queue[3];
  if ((uint64_t)blockIdx.x * blockDim.x >= count) return;  // the same for the whole CTA
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Smem sm;
  uint32_t* lut = reinterpret_cast<uint32_t*>(smem);
  const uint16_t* syms = reinterpret_cast<const uint16_t*>(s + h.L.table + 4 * (kMaxLen + 1));
  if (!cta_tables(s, h, sm, lut, syms, st)) return;
  __syncthreads();
  const Tables tb = {lut, &sm.cn, syms, h.n_live, nullptr, 0u, 0u};
  Walker<T, 3> wk;
  wk.base = reinterpret_cast<T*>(smem + (4u << kLutBits)) + threadIdx.x;
  wk.stride = blockDim.x;
  wk.B2 = h.g.B[2];
  wk.sr = h.g.B[1] * h.g.B[2];
  Acc acc;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = dw.fix[idx];
    BlockIn bi;
    uint8_t stv;
    if (!place_block(s, h, b, &bi)) {
      stv = SDCSZ_BLOCK_BAD;
      ++acc.bad;
    } else {
      unsigned long long sum = 0, nv = 0;
      double me = 0.0;
      const bool ok = decode_generic<T, 3>(s, s + nbytes, h, bi, tb, wk, FieldSink<T>{field}, nullptr, kNone, 0, &sum,
                                           &nv, &me);
      if (ok && sum == ld_u64(s + h.L.sumdc + 8 * b)) {
        stv = SDCSZ_BLOCK_CORRECTED;
        ++acc.fix;
      } else {
        stv = ok ? SDCSZ_BLOCK_SDC : SDCSZ_BLOCK_BAD;
        ++acc.bad;
      }
    }
    if (status) status[b] = stv;
  }
  acc.commit(st);
}

template <typename T, int B, int G, bool CMP>
void run_wave_decode(const uint8_t* s, uint64_t nbytes, const Hdr& h, T* field, uint8_t* status, State* st,
                     uint8_t* wave_ws, const Launch& L) {
  typedef DWaveCfg<T, B, G> C;
  const DWs dw = bind_dws(wave_ws, h.g);
  {
    const size_t smem = 12u << kLutBits;  // lut and pair lut
    auto ka = k_wave_codes<T, B, CMP>;
    const unsigned grid = persistent_grid(ka, 256, smem, (h.g.nb + 255) / 256, L);
    ka<<<grid, 256, smem, L.stream>>>(s, nbytes, h, st, dw);
    note_launch();
  }
  {
    auto kb = k_wave_recon<T, B, G, CMP>;
    const uint64_t items = (h.g.nb + G - 1) / G + (edge_count(h.g) + G - 1) / G;
    const unsigned grid = persistent_grid(kb, C::NT, C::SMEM, items, L);
    kb<<<grid, C::NT, C::SMEM, L.stream>>>(s, h, field, status, st, dw);
    note_launch();
  }
  if (h.g.abft) {
    const size_t smem = (4u << kLutBits) + (size_t)walker_slots(3, h.g.B) * 64 * sizeof(T);
    auto kc = k_wave_fixup<T>;
    allow_smem(reinterpret_cast<const void*>(kc), smem);
    kc<<<2 * L.sms, 64, smem, L.stream>>>(s, nbytes, h, field, status, st, dw);
    note_launch();
  }
}

// The two-pass decoder for the shapes it serves (3D cubes of edge 10, 12, 16), false otherwise.
template <typename T, bool CMP>
bool try_wave_decode(const uint8_t* s, uint64_t nbytes, const Hdr& h, T* field, uint8_t* status, State* st,
                     uint8_t* wave_ws, const Launch& L) {
  const Geo& g = h.g;
  if (g.ndim != 3 || g.B[0] != g.B[1] || g.B[1] != g.B[2] || !g.nb) return false;
  switch (g.B[2]) {
    case 10: run_wave_decode<T, 10, 16, CMP>(s, nbytes, h, field, status, st, wave_ws, L); return true;
    case 12: run_wave_decode<T, 12, 16, CMP>(s, nbytes, h, field, status, st, wave_ws, L); return true;
    case 16: run_wave_decode<T, 16, 8, CMP>(s, nbytes, h, field, status, st, wave_ws, L); return true;
    default: return false;
  }
}

}  // namespace
}  // namespace kdec
}  // namespace sdcsz
