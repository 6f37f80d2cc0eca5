// K5: fault-tolerant decompression (Alg. 2 of the paper, without the Zstd stage).
//
// Persistent CTAs, each taking whole random-access groups of 256 blocks; one thread per
// block. A CTA builds a 12-bit first-level decode table for the canonical Huffman code in
// shared memory (longer codes resolve through the canonical first-code table), scans the
// group's block table for per-block offsets and checks the group table against it. Each
// thread then decodes its block and reconstructs it with the Lorenzo or regression predictor
// (the decompression loop of Algorithm 2). For fault-tolerant streams the block's checksum is
// compared with sum_dc; on a mismatch the block is decompressed once more from its compressed
// bytes (random-access re-execution) and reported corrected or as an SDC in compression.
// As in compression, full blocks of the common shapes take a fast kernel with compile-time
// edges and edge blocks a generic kernel. In the compact encoding a regression block's
// payload starts with its coefficient integers and each code 0 is followed by the point's
// truncated value.
#pragma once

#include <algorithm>
#include <type_traits>

#include "sdcsz_internal.cuh"

namespace sdcsz {
namespace kdec {
namespace {

constexpr uint32_t kNone = 0xffffffffu;
constexpr int kDefer = -2;  // second symbol of a pair not decoded yet (compact encoding: a value comes first)

struct Canon {
  uint32_t fc[kMaxLen + 2];  // first code of each length
  uint32_t fi[kMaxLen + 2];  // canonical index of that first code
  uint32_t nc[kMaxLen + 2];  // codes of each length
  uint32_t bins;             // symbols must be below this
};

__device__ __forceinline__ unsigned long long ld_u64(const uint8_t* p) {
  return *reinterpret_cast<const unsigned long long*>(p);
}

__device__ __forceinline__ void mad_wide(unsigned long long& acc, uint32_t a, uint32_t b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

template <typename T>
__device__ __forceinline__ void sum_words(T v, unsigned long long& sum) {
  mad_wide(sum, FT<T>::lo(v), 1u);
  if (FT<T>::W == 2) mad_wide(sum, FT<T>::hi(v), 1u);
}

// Long codes (> 12 bits) through the canonical tables; returns the symbol or -1.
__device__ __noinline__ int slow_symbol(unsigned long long buf, const Canon& cn, const uint16_t* syms,
                                        uint32_t n_live, uint32_t* len_out) {
  for (uint32_t l = kLutBits + 1; l <= (uint32_t)kMaxLen; ++l) {
    const uint32_t c = (uint32_t)(buf >> (64 - l));
    if (c - cn.fc[l] < cn.nc[l]) {
      const uint32_t r = cn.fi[l] + (c - cn.fc[l]);
      if (r >= n_live || syms[r] >= cn.bins) return -1;
      *len_out = l;
      return syms[r];
    }
  }
  return -1;
}

// MSB-first bit reader fed by aligned 32-bit words; never reads at or past `lim`.
struct BitReader {
  const uint8_t* wp;   // next aligned word
  const uint8_t* lim;  // end of the stream
  unsigned long long buf;
  int nb;
  uint32_t used;
  __device__ __forceinline__ uint32_t word() {
    uint32_t w;
    if (wp + 4 <= lim) {
      w = __byte_perm(__ldg(reinterpret_cast<const uint32_t*>(wp)), 0, 0x0123);
    } else {
      w = 0;
      for (int q = 0; q < 4; ++q) w |= (wp + q < lim ? (uint32_t)wp[q] : 0u) << (24 - 8 * q);
    }
    wp += 4;
    return w;
  }
  __device__ __forceinline__ void init(const uint8_t* p, const uint8_t* end) {
    lim = end;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    wp = reinterpret_cast<const uint8_t*>(a & ~uintptr_t(3));
    const int skip = (int)(a & 3) * 8;
    buf = (unsigned long long)word() << 32;
    buf |= word();
    buf <<= skip;
    nb = 64 - skip;
    used = 0;
  }
  // the next n (1..32) raw bits
  __device__ __forceinline__ uint32_t bits(uint32_t n) {
    if (nb <= 32) {
      buf |= (unsigned long long)word() << (32 - nb);
      nb += 32;
    }
    const uint32_t v = (uint32_t)(buf >> (64 - n));
    buf <<= n;
    nb -= (int)n;
    used += n;
    return v;
  }
  // next symbol, or -1 for an invalid code
  __device__ __forceinline__ int next(const uint32_t* lut, const Canon& cn, const uint16_t* syms, uint32_t n_live) {
    if (nb <= 32) {
      buf |= (unsigned long long)word() << (32 - nb);
      nb += 32;
    }
    const uint32_t e = lut[buf >> (64 - kLutBits)];
    uint32_t len = e & 0xffu;
    int sym;
    if (len) {
      sym = (int)(e >> 8);
    } else {
      sym = slow_symbol(buf, cn, syms, n_live, &len);
      if (sym < 0) return -1;
    }
    buf <<= len;
    nb -= (int)len;
    used += len;
    return sym;
  }
};

// Unchecked variant for payloads far enough from the end of the stream (the caller checks
// the worst case). Two big-endian words w0:w1 hold the next 64 bits from bit `pos` of w0; a
// symbol is a 12-bit table lookup on a funnel shift, and crossing into the next word is
// predicated rather than branched (lanes cross at different symbols).
struct FastReader {
  const uint32_t* wp;  // next word to prefetch
  const uint32_t* w_start;
  uint32_t w0, w1, w2, pos, skip;  // w2: the word after w1, loaded ahead of use
  __device__ __forceinline__ void init(const uint8_t* p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    wp = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
    w_start = wp;
    w0 = __byte_perm(__ldg(wp), 0, 0x0123);
    w1 = __byte_perm(__ldg(wp + 1), 0, 0x0123);
    w2 = __ldg(wp + 2);
    wp += 3;
    skip = pos = (uint32_t)(a & 3) * 8;
  }
  // bits consumed since init
  __device__ __forceinline__ uint32_t used() const { return (uint32_t)(wp - w_start - 3) * 32u + pos - skip; }
  __device__ __forceinline__ int next(const uint32_t* lut, const Canon& cn, const uint16_t* syms, uint32_t n_live) {
    const uint32_t peek = __funnelshift_l(w1, w0, pos);
    const uint32_t e = lut[peek >> (32 - kLutBits)];
    uint32_t len = e & 0xffu;
    int sym = (int)(e >> 8);
    if (!len) {
      sym = slow_symbol((unsigned long long)peek << 32, cn, syms, n_live, &len);
      if (sym < 0) return -1;
    }
    advance(len);
    return sym;
  }
  // the next 32 bits, not consumed
  __device__ __forceinline__ uint32_t peek() const { return __funnelshift_l(w1, w0, pos); }
  // the next n (1..32) raw bits
  __device__ __forceinline__ uint32_t bits(uint32_t n) {
    const uint32_t peek = __funnelshift_l(w1, w0, pos);
    advance(n);
    return n == 32 ? peek : peek >> (32 - n);
  }
  __device__ __forceinline__ void advance(uint32_t len) {
    pos += len;
    if (pos >= 32) {  // only lanes crossing a word boundary touch memory
      pos -= 32;
      w0 = w1;
      w1 = __byte_perm(w2, 0, 0x0123);
      w2 = __ldg(wp);
      ++wp;
    }
  }
  // Two symbols with one lookup when both codes lie in the 12-bit window (the pair table
  // holds the second symbol only then), else one at a time. In the compact encoding a code 0
  // is followed by its value, so after a first symbol 0 the second is left for later (kDefer).
  __device__ __forceinline__ void next2(const uint2* lut2, const uint32_t* lut, const Canon& cn, const uint16_t* syms,
                                        uint32_t n_live, int& q0, int& q1, bool compact) {
    const uint32_t peek = __funnelshift_l(w1, w0, pos);
    const uint2 e = lut2[peek >> (32 - kLutBits)];
    const uint32_t l0 = e.x & 0xffu, l1 = e.y & 0xffu;
    if (l1) {
      q0 = (int)(e.x >> 8);
      q1 = (int)(e.y >> 8);
      advance(l0 + l1);
    } else {
      q0 = next(lut, cn, syms, n_live);
      q1 = (compact && q0 == 0) ? kDefer : next(lut, cn, syms, n_live);
    }
  }
};

// Compact encoding: one coefficient integer (bit length of its zigzag value in 6 bits, then the
// bits below the leading one); false for a length above 32.
template <class Reader>
__device__ __forceinline__ bool read_coef(Reader& br, int* k) {
  const uint32_t n = br.bits(6);
  if (n > 32) return false;
  uint32_t z = 0;
  if (n > 0) z = (n > 1 ? br.bits(n - 1) : 0u) | (1u << (n - 1));
  *k = (int)((z >> 1) ^ (0u - (z & 1u)));
  return true;
}

// Compact encoding: one unpredictable value (sign and exponent, then the kept mantissa bits).
template <typename T, class Reader>
__device__ __forceinline__ T read_unpred(Reader& br, int texp) {
  typedef typename Bitsof<T>::U U;
  const uint32_t se = br.bits(1 + Bitsof<T>::E);
  const int Ex = (int)(se & ((1u << Bitsof<T>::E) - 1));
  int m = Bitsof<T>::M;
  if (Ex != 0 && Ex != (1 << Bitsof<T>::E) - 1) m = min(max(Ex - Bitsof<T>::BIAS - texp, 0), Bitsof<T>::M);
  U mant = 0;
  if (m > 32) {  // float64 only (a float keeps at most 23 bits)
    mant = (U)((unsigned long long)br.bits((uint32_t)m - 32) << 32);
    mant |= br.bits(32);
  } else if (m > 0) {
    mant = br.bits((uint32_t)m);
  }
  return Bitsof<T>::val(((U)se << Bitsof<T>::M) | (mant << (Bitsof<T>::M - m)));
}

// The coefficients of a regression block: stored dtype values, or (compact encoding) the
// integers at the head of its payload times their steps.
template <typename T, int NDIM, class Reader>
__device__ __forceinline__ bool block_coefs(const uint8_t* s, const Hdr& h, int64_t reg_idx, Reader& br, T cT[4],
                                            bool compact) {
  if (compact) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a <= NDIM; ++a) {
      int k = 0;
      if (ok) ok = read_coef(br, &k);
      cT[a] = coef_from_int<T>(k, h.cstep[a]);
    }
    return ok;
  }
  const T* c = reinterpret_cast<const T*>(s + h.L.coef) + (uint64_t)(NDIM + 1) * reg_idx;
#pragma unroll
  for (int a = 0; a <= NDIM; ++a) cT[a] = c[a];
  return true;
}

struct BlockIn {
  uint64_t b, pay_off, un_off;
  uint32_t size, ucnt;
  int64_t reg_idx;
};

struct Tables {
  const uint32_t* lut;
  const Canon* cn;
  const uint16_t* syms;
  uint32_t n_live;
  const uint2* lut2;  // pair table (fast decoder only)
  // fast decoder only: a row of central codes (prediction within half a bin) is the central
  // codeword repeated, rpat, rbits bits long; rbits = 0 when that does not fit a word
  uint32_t rbits, rpat;
};

// Pair table: entry p holds lut[p] and, when that code is shorter than the window and the
// code after it also ends inside the window, that second code's lut entry (else 0). Only the
// window's known bits decide either symbol. In the compact encoding a code 0 is followed by a
// value, not a code, so it never starts a pair. Call after the lut is complete and visible.
__device__ __forceinline__ void pair_table(uint2* lut2, const uint32_t* lut, bool compact) {
  for (uint32_t e = threadIdx.x; e < (1u << kLutBits); e += blockDim.x) {
    const uint32_t v1 = lut[e], l1 = v1 & 0xffu;
    uint32_t v2 = 0;
    if (l1 && l1 < (uint32_t)kLutBits && !(compact && (v1 >> 8) == 0)) {
      const uint32_t u = lut[(e << l1) & ((1u << kLutBits) - 1)], l2 = u & 0xffu;
      if (l2 && l2 <= (uint32_t)kLutBits - l1) v2 = u;
    }
    lut2[e] = make_uint2(v1, v2);
  }
}

// ---------------------------------------------------------------- generic path
// Where the generic decoder stores a block's values: the whole field (or nowhere when
// verifying), or a dense sub-box of the field (region decompression).
template <typename T>
struct FieldSink {
  T* field;
  __device__ __forceinline__ T* row(const Geo& g, const Box& x, uint32_t i, uint32_t j) const {
    return field ? field + row_base(g, x, i, j) : nullptr;
  }
  __device__ __forceinline__ bool col(const Box&, uint32_t) const { return true; }
};

template <typename T>
struct RegionSink {
  T* out;
  uint64_t lo[3], hi[3];  // the box in padded 3D coordinates, [lo, hi)
  // element l of the block row is at row(...)[l] (dereferenced only where col() holds)
  __device__ __forceinline__ T* row(const Geo&, const Box& x, uint32_t i, uint32_t j) const {
    const uint64_t gi = x.org[0] + i, gj = x.org[1] + j;
    if (gi < lo[0] || gi >= hi[0] || gj < lo[1] || gj >= hi[1]) return nullptr;
    const int64_t r = (int64_t)(((gi - lo[0]) * (hi[1] - lo[1]) + (gj - lo[1])) * (hi[2] - lo[2]));
    return out + (r + ((int64_t)x.org[2] - (int64_t)lo[2]));
  }
  __device__ __forceinline__ bool col(const Box& x, uint32_t l) const {
    const uint64_t gl = x.org[2] + l;
    return gl >= lo[2] && gl < hi[2];
  }
};

template <typename T, int NDIM, class Sink = FieldSink<T>>
__device__ __noinline__ bool decode_generic(const uint8_t* __restrict__ s, const uint8_t* lim, const Hdr& h,
                                            const BlockIn& bi, const Tables& tb, Walker<T, NDIM>& wk,
                                            const Sink sink, const T* __restrict__ orig, uint32_t kinj,
                                            uint32_t bitinj, unsigned long long* sum_out, unsigned long long* viol,
                                            double* maxerr) {
  const Geo& g = h.g;
  const Box x = block_box(g, bi.b);
  const T eb = (T)h.eb;
  T cT[4] = {T(0), T(0), T(0), T(0)};
  const bool reg = bi.reg_idx >= 0;
  const T* un = reinterpret_cast<const T*>(s + h.L.unpred) + bi.un_off;
  BitReader br;
  br.init(s + h.L.payload + bi.pay_off, lim);
  bool ok = true;
  if (reg) ok = block_coefs<T, NDIM>(s, h, bi.reg_idx, br, cT, h.g.enc != 0);
  uint32_t used_u = 0, k = 0;
  unsigned long long sum = 0, nv = 0;
  double me = 0.0;
  for (uint32_t i = 0; i < x.e[0]; ++i) {
    for (uint32_t j = 0; j < x.e[1]; ++j) {
      const uint64_t rb = row_base(g, x, i, j);
      T* dst = sink.row(g, x, i, j);
      wk.row_start();
      for (uint32_t l = 0; l < x.e[2]; ++l, ++k) {
        const int q = ok ? br.next(tb.lut, *tb.cn, tb.syms, tb.n_live) : -1;
        T xr = T(0);
        if (!reg) wk.load(i, j, l);
        if (q < 0 || (uint32_t)q >= g.bins) {
          ok = false;
        } else if (q == 0) {
          if (used_u >= bi.ucnt) ok = false;
          else if (h.g.enc) xr = read_unpred<T>(br, h.texp);
          else xr = un[used_u];
          ++used_u;
        } else {
          const T pred = reg ? regress<T, NDIM, OpRN<T>>(cT, i, j, l) : wk.template combine<OpRN<T>>();
          xr = FT<T>::add(pred, FT<T>::mul(FT<T>::fromi(2 * (q - (int)g.R)), eb));
        }
        if (k == kinj) xr = FT<T>::flip(xr, bitinj);
        if (!reg) wk.commit(j, l, xr);
        if (dst && sink.col(x, l)) dst[l] = xr;
        if (orig) {
          const T xo = orig[rb + l];
          bool bad;
          if (FT<T>::finite(xo)) {
            const T d = FT<T>::absv(FT<T>::sub(xo, xr));
            bad = !(d <= eb);
            if (!bad) me = fmax(me, (double)d);
          } else {
            bad = !FT<T>::same(xo, xr);
          }
          nv += bad;
        }
        sum_words<T>(xr, sum);
      }
    }
  }
  if (used_u != bi.ucnt || br.used > bi.size * 8u) ok = false;
  *sum_out = sum;
  *viol = nv;
  *maxerr = me;
  return ok;
}

// ---------------------------------------------------------------- fast path (full blocks)
// WRITE: decompression (the block is stored to blk_out); otherwise verification (compared
// with blk_orig when there is one). EDGE: a block cut by the field boundary, extents
// e0 x e1 x e2 within the compile-time shape: the loops stop at the extents, a central row is
// e2 central codewords, symbols are decoded one at a time and stored one at a time.
template <typename T, int NDIM, int B0, int B1, int B2, bool REG, bool HOOK, bool WRITE, bool CMP, bool EDGE = false>
__device__ __forceinline__ bool decode_fast(const uint8_t* __restrict__ s, const uint8_t* lim, const Hdr& h,
                                            const BlockIn& bi, const Tables& tb, T* plane, T* __restrict__ blk_out,
                                            const T* __restrict__ blk_orig, uint64_t si, uint64_t sj, bool vec2,
                                            uint32_t kinj, uint32_t bitinj, unsigned long long* sum_out,
                                            unsigned long long* viol, double* maxerr, uint32_t e0 = B0,
                                            uint32_t e1 = B1, uint32_t e2 = B2) {
  const Geo& g = h.g;
  const T eb = (T)h.eb;
  const int R = (int)g.R;
  T cT[4] = {T(0), T(0), T(0), T(0)};
  const T* un = reinterpret_cast<const T*>(s + h.L.unpred) + bi.un_off;
  FastReader br;
  br.init(s + h.L.payload + bi.pay_off);
  (void)lim;
  bool ok = true;
  if (REG) ok = block_coefs<T, NDIM>(s, h, bi.reg_idx, br, cT, CMP);
  uint32_t used_u = 0;
  unsigned long long sum = 0, nv = 0;
  double me = 0.0;
  if (!REG && NDIM == 3) {
#pragma unroll
    for (int q = 0; q < B1 * B2; ++q) plane[q * 256] = T(0);
  }
  // regression along the row: the block's products c_l * l
  T clp[B2];
  if (REG) {
#pragma unroll
    for (int l = 0; l < B2; ++l) clp[l] = FT<T>::mul(cT[NDIM == 3 ? 2 : 1], (T)l);
  }
  // a central row: the central codeword repeated over the row (e2 codes for an edge block)
  uint32_t rbits = tb.rbits, rpat = tb.rpat;
  if (EDGE && rbits) {
    const uint32_t lc = rbits / B2;
    rbits = lc * e2;
    rpat >>= lc * (B2 - e2);
  }
  const int n0 = EDGE ? (int)e0 : B0, n1 = EDGE ? (int)e1 : B1;
  T brow[B2], arow[B2];
#pragma unroll 1
  for (int i = 0; i < n0; ++i) {
#pragma unroll
    for (int l = 0; l < B2; ++l) {
      brow[l] = T(0);
      arow[l] = T(0);
    }
#pragma unroll 1
    for (int j = 0; j < n1; ++j) {
      T ra = T(0);
      if (REG) {
        if (NDIM == 3) ra = FT<T>::add(FT<T>::mul(cT[0], (T)i), FT<T>::mul(cT[1], (T)j));
        else ra = FT<T>::mul(cT[0], (T)j);
      }
      T* prow = plane + j * B2 * 256;
      T out[B2];
      T c = T(0), ac = T(0), bc = T(0), abc = T(0);
      const uint32_t k0 = EDGE ? (uint32_t)((i * n1 + j) * (int)e2) : (uint32_t)((i * B1 + j) * B2);
      // the neighbours of point l (Lorenzo) and its prediction
      auto predict = [&](int l, T& a, T& bb, T& ab) {
        a = bb = ab = T(0);
        if (REG) {
          if (NDIM == 3) return FT<T>::add(FT<T>::add(ra, clp[l]), cT[3]);
          return FT<T>::add(FT<T>::add(ra, clp[l]), cT[2]);
        }
        if (NDIM == 3) {
          a = prow[l * 256];
          bb = brow[l];
          ab = arow[l];
          T sacc = FT<T>::add(a, bb);
          sacc = FT<T>::sub(sacc, ab);
          sacc = FT<T>::sub(sacc, ac);
          sacc = FT<T>::sub(sacc, bc);
          sacc = FT<T>::add(sacc, abc);
          return FT<T>::add(sacc, c);
        }
        a = brow[l];
        return FT<T>::add(FT<T>::sub(a, ac), c);
      };
      // point l reconstructed as xr: the Lorenzo state, the output row and sum_dc
      auto commit = [&](int l, T xr, T a, T bb, T ab) {
        if (HOOK && k0 + l == kinj) xr = FT<T>::flip(xr, bitinj);
        if (!REG) {
          if (NDIM == 3) {
            prow[l * 256] = xr;
            arow[l] = a;
            ac = a;
            bc = bb;
            abc = ab;
          } else {
            ac = a;
          }
          brow[l] = xr;
          c = xr;
        }
        out[l] = xr;
        sum_words<T>(xr, sum);
      };
      // a row of central codes (the common case of a smooth field) in one comparison: every
      // point is pred + (T)(2 * 0) * eb = pred + 0
      if (rbits && (br.peek() >> (32 - rbits)) == rpat) {
        br.advance(rbits);
#pragma unroll
        for (int l = 0; l < B2; ++l) {
          if (EDGE && l >= (int)e2) break;
          T a, bb, ab;
          const T pred = predict(l, a, bb, ab);
          commit(l, FT<T>::add(pred, T(0)), a, bb, ab);
        }
      } else {
        int qp = 0;  // second symbol of the pair decoded at even l
#pragma unroll
        for (int l = 0; l < B2; ++l) {
          if (EDGE && l >= (int)e2) break;
          int q;
          if (!EDGE && (B2 & 1) == 0) {  // the fast shapes have even rows: symbols come in pairs
            if (!(l & 1)) br.next2(tb.lut2, tb.lut, *tb.cn, tb.syms, tb.n_live, q, qp, CMP);
            else q = (CMP && qp == kDefer) ? br.next(tb.lut, *tb.cn, tb.syms, tb.n_live) : qp;
          } else {
            q = br.next(tb.lut, *tb.cn, tb.syms, tb.n_live);
          }
          T a, bb, ab;
          const T pred = predict(l, a, bb, ab);
          T xr = FT<T>::add(pred, FT<T>::mul(FT<T>::fromi(2 * (q - R)), eb));
          if (q <= 0) {  // unpredictable value (code 0) or an undecodable block (rare)
            xr = T(0);
            if (q == 0 && used_u < bi.ucnt) xr = CMP ? read_unpred<T>(br, h.texp) : un[used_u];
            else ok = false;
            ++used_u;
          }
          commit(l, xr, a, bb, ab);
        }
      }
      const uint64_t ro = (uint64_t)i * si + (uint64_t)j * sj;
      if (WRITE) {  // streaming stores: the field is not read again, the stream's bytes are
        if (EDGE) {
#pragma unroll
          for (int l = 0; l < B2; ++l)
            if (l < (int)e2) __stcs(blk_out + ro + l, out[l]);
        } else if ((B2 % 2) == 0 && vec2) {
          typedef typename std::conditional<sizeof(T) == 4, float2, double2>::type V2;
          V2* p = reinterpret_cast<V2*>(blk_out + ro);
#pragma unroll
          for (int l = 0; l < B2 / 2; ++l) {
            V2 t;
            t.x = out[2 * l];
            t.y = out[2 * l + 1];
            __stcs(p + l, t);
          }
        } else {
#pragma unroll
          for (int l = 0; l < B2; ++l) __stcs(blk_out + ro + l, out[l]);
        }
      }
      if (!WRITE && blk_orig) {
#pragma unroll
        for (int l = 0; l < B2; ++l) {
          if (EDGE && l >= (int)e2) break;
          const T xo = blk_orig[ro + l];
          bool bad;
          if (FT<T>::finite(xo)) {
            const T d = FT<T>::absv(FT<T>::sub(xo, out[l]));
            bad = !(d <= eb);
            if (!bad) me = fmax(me, (double)d);
          } else {
            bad = !FT<T>::same(xo, out[l]);
          }
          nv += bad;
        }
      }
    }
  }
  if (used_u != bi.ucnt || br.used() > bi.size * 8u) ok = false;
  *sum_out = sum;
  *viol = nv;
  *maxerr = me;
  return ok;
}

// ---------------------------------------------------------------- CTA set-up and group scan
struct Smem {
  Canon cn;
  uint32_t sz[kGroup], uc[kGroup], rg[kGroup];
  unsigned long long off[kGroup][3];
  unsigned long long wt[8][3];
  int bad;
};

// Canonical tables (validated) and the first-level decode table; false for a bad code table.
__device__ bool cta_tables(const uint8_t* s, const Hdr& h, Smem& sm, uint32_t* lut, const uint16_t* syms,
                           State* st) {
  if (threadIdx.x == 0) {
    const uint32_t* blc = reinterpret_cast<const uint32_t*>(s + h.L.table);
    unsigned long long kraft = 0, total = 0;
    uint32_t code = 0, idx = 0;
    int bad = blc[0] != 0;
    for (uint32_t l = 1; l <= (uint32_t)kMaxLen; ++l) {
      const uint32_t c = blc[l];
      code = (code + (l >= 2 ? sm.cn.nc[l - 1] : 0u)) << 1;
      sm.cn.fc[l] = code;
      sm.cn.fi[l] = idx;
      sm.cn.nc[l] = c;
      idx += c;
      kraft += (unsigned long long)c << (kMaxLen - l);
      total += c;
    }
    if (total != h.n_live || kraft > (1ull << kMaxLen)) bad = 1;
    sm.cn.bins = h.g.bins;
    sm.bad = bad;
    if (bad) atomicOr(&st->error, ERR_FORMAT);
  }
  __syncthreads();
  if (sm.bad) return false;
  for (uint32_t e = threadIdx.x; e < (1u << kLutBits); e += blockDim.x) {
    uint32_t v = 0;
    for (uint32_t l = 1; l <= (uint32_t)kLutBits; ++l) {
      const uint32_t c = e >> (kLutBits - l);
      if (c - sm.cn.fc[l] < sm.cn.nc[l]) {
        const uint32_t r = sm.cn.fi[l] + (c - sm.cn.fc[l]);
        const uint32_t sym = r < h.n_live ? syms[r] : 0xffffffffu;
        v = sym < h.g.bins ? ((sym << 8) | l) : 0u;  // an out-of-range symbol decodes as invalid
        break;
      }
    }
    lut[e] = v;
  }
  return true;
}

// Offsets of the group's blocks; false (and a format error) when the stored group bases
// disagree with the block table.
__device__ bool group_scan(const uint8_t* s, const Hdr& h, uint64_t gid, uint64_t ngroups, Smem& sm, State* st) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const Geo& g = h.g;
  const uint64_t b0 = gid * kGroup;
  const uint32_t nblk = (uint32_t)min((uint64_t)kGroup, g.nb - b0);
  __syncthreads();
  for (uint32_t t = tid; t < kGroup; t += blockDim.x) {
    const uint64_t b = b0 + t;
    const bool in = t < nblk;
    sm.sz[t] = in ? *reinterpret_cast<const uint16_t*>(s + h.L.sizes + 2 * b) : 0u;
    sm.uc[t] = in ? *reinterpret_cast<const uint16_t*>(s + h.L.ucounts + 2 * b) : 0u;
    sm.rg[t] = in ? ((*reinterpret_cast<const uint32_t*>(s + h.L.bitmap + 4 * (b / 32)) >> (b % 32)) & 1u) : 0u;
  }
  __syncthreads();
  const uint32_t R = kGroup / blockDim.x;
  unsigned long long loc[3] = {0, 0, 0};
  for (uint32_t r = 0; r < R; ++r) {
    const uint32_t e = tid * R + r;
    loc[0] += sm.sz[e];
    loc[1] += sm.uc[e];
    loc[2] += sm.rg[e];
  }
  unsigned long long inc[3] = {loc[0], loc[1], loc[2]};
  for (int o = 1; o < 32; o <<= 1)
    for (int q = 0; q < 3; ++q) {
      const unsigned long long n = __shfl_up_sync(0xffffffffu, inc[q], o);
      if (lane >= (uint32_t)o) inc[q] += n;
    }
  if (lane == 31)
    for (int q = 0; q < 3; ++q) sm.wt[wid][q] = inc[q];
  __syncthreads();
  if (tid == 0) {
    unsigned long long run[3] = {0, 0, 0};
    for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2)
      for (int q = 0; q < 3; ++q) {
        const unsigned long long t = sm.wt[w2][q];
        sm.wt[w2][q] = run[q];
        run[q] += t;
      }
    const uint8_t* gp = s + h.L.groups + 24 * gid;
    unsigned long long base[3] = {ld_u64(gp), ld_u64(gp + 8), ld_u64(gp + 16)}, next[3];
    if (gid + 1 < ngroups) {
      next[0] = ld_u64(gp + 24);
      next[1] = ld_u64(gp + 32);
      next[2] = ld_u64(gp + 40);
    } else {
      next[0] = h.payload_bytes;
      next[1] = h.n_unpred;
      next[2] = h.n_reg;
    }
    int bad = 0;
    for (int q = 0; q < 3; ++q) bad |= (base[q] + run[q] != next[q]) || (gid == 0 && base[q] != 0);
    sm.bad = bad;
    if (bad) atomicOr(&st->error, ERR_FORMAT);
    for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2)
      for (int q = 0; q < 3; ++q) sm.wt[w2][q] += base[q];
  }
  __syncthreads();
  unsigned long long run[3];
  for (int q = 0; q < 3; ++q) run[q] = sm.wt[wid][q] + inc[q] - loc[q];
  for (uint32_t r = 0; r < R; ++r) {
    const uint32_t e = tid * R + r;
    sm.off[e][0] = run[0];
    sm.off[e][1] = run[1];
    sm.off[e][2] = run[2];
    run[0] += sm.sz[e];
    run[1] += sm.uc[e];
    run[2] += sm.rg[e];
  }
  __syncthreads();
  return !sm.bad;
}

// Group gid's data on its way to L2, a group ahead of its decoding: its block-table, unpredictable-count
// and sum_dc entries (fixed places; a line per thread) and, by warp 0 after reading the group
// table, its payload and coefficient ranges. Every address is clamped to the stream.
__device__ __forceinline__ void prefetch_group(const uint8_t* s, uint64_t nbytes, const Hdr& h, uint64_t gid,
                                               uint64_t ngroups) {
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint64_t b0 = gid * kGroup;
  {
    uint64_t off;
    if (tid < 4) off = h.L.sizes + 2 * b0 + 128 * tid;
    else if (tid < 8) off = h.L.ucounts + 2 * b0 + 128 * (tid - 4);
    else if (tid < 24 && h.g.abft) off = h.L.sumdc + 8 * b0 + 128 * (tid - 8);
    else off = nbytes;
    if (off < nbytes) prefetch_l2(s + off);
  }
  if (tid >= 32) return;
  const uint8_t* gp = s + h.L.groups + 24 * gid;
  const uint64_t p0 = ld_u64(gp), r0 = ld_u64(gp + 16);
  const bool last = gid + 1 >= ngroups;
  const uint64_t p1 = last ? h.payload_bytes : ld_u64(gp + 24), r1 = last ? h.n_reg : ld_u64(gp + 40);
  auto range = [&](uint64_t lo, uint64_t hi, uint64_t floor_, uint64_t ceil_) {
    lo = max(lo, floor_);
    hi = min(min(hi, ceil_), lo + 65536);  // a group's payload rarely exceeds a few KB
    for (uint64_t a = (lo & ~uint64_t(127)) + 128 * (uint64_t)lane; a < hi; a += 32 * 128) prefetch_l2(s + a);
  };
  if (p0 <= p1) range(h.L.payload + p0, h.L.payload + p1, h.L.payload, nbytes);
  const uint64_t cs = (uint64_t)(h.g.ndim + 1) * (h.g.dtype ? 8 : 4);
  if (!h.g.enc && r0 <= r1 && r1 <= h.n_reg) range(h.L.coef + cs * r0, h.L.coef + cs * r1, h.L.coef, nbytes);
}

struct Acc {
  unsigned long long fix = 0, bad = 0, viol = 0;
  double maxerr = 0.0;
  __device__ __forceinline__ void commit(State* st) {
    fix = warp_sum(fix);
    bad = warp_sum(bad);
    viol = warp_sum(viol);
    for (int o = 16; o > 0; o >>= 1) maxerr = fmax(maxerr, __shfl_xor_sync(0xffffffffu, maxerr, o));
    if ((threadIdx.x & 31) == 0) {
      if (fix) atomicAdd(&st->reexec_corrected, fix);
      if (bad) atomicAdd(&st->uncorrectable, bad);
      if (viol) atomicAdd(&st->bound_viol, viol);
      if (maxerr > 0.0) atomicMax(&st->max_err_bits, (unsigned long long)__double_as_longlong(maxerr));
    }
  }
};

__device__ __forceinline__ bool is_full(const Geo& g, uint64_t b) {
  uint64_t c0, c1, c2;
  block_coords(g, b, c0, c1, c2);
  return (c0 + 1) * g.B[0] <= g.d[0] && (c1 + 1) * g.B[1] <= g.d[1] && (c2 + 1) * g.B[2] <= g.d[2];
}

// Algorithm 2's verification around one decode: check against sum_dc, re-execute once.
template <class F>
__device__ __forceinline__ uint8_t verify_block(const uint8_t* s, const Hdr& h, uint64_t b, F run, Acc& acc) {
  unsigned long long sum = 0, nv = 0;
  double me = 0.0;
  // the stored sum_dc is loaded before the block is decoded, so the load is in flight meanwhile
  const unsigned long long ref = h.g.abft ? ld_u64(s + h.L.sumdc + 8 * b) : 0ull;
  bool ok = run(true, &sum, &nv, &me);
  uint8_t stv = SDCSZ_BLOCK_OK;
  if (h.g.abft) {
    if (!ok || sum != ref) {
      ok = run(false, &sum, &nv, &me);  // decompress this block again from its bytes
      if (ok && sum == ref) {
        stv = SDCSZ_BLOCK_CORRECTED;
        ++acc.fix;
      } else {
        stv = ok ? SDCSZ_BLOCK_SDC : SDCSZ_BLOCK_BAD;
        ++acc.bad;
      }
    }
  } else if (!ok) {
    stv = SDCSZ_BLOCK_BAD;
    ++acc.bad;
  }
  acc.viol += nv;
  acc.maxerr = fmax(acc.maxerr, me);
  return stv;
}

__device__ __forceinline__ void find_inj(const sdcsz_flip* flips, uint32_t nflips, uint64_t b, uint32_t* k,
                                         uint32_t* bit) {
  *k = kNone;
  *bit = 0;
  uint64_t idx;
  if (nflips && find_flip(flips, nflips, SDCSZ_SITE_DECOMP, b, &idx, bit)) *k = (uint32_t)min(idx, (uint64_t)kNone - 1);
}

// The payload, unpredictable and coefficient offsets of block b from its group's table entry
// plus the block-table entries before it in the group: eight 16-bit entries per 16-byte load
// (the sections are 16-byte aligned and a group starts at a multiple of 256 entries) and the
// regression flags by whole bitmap words. False when the entries point outside the stream.
__device__ __forceinline__ bool place_block(const uint8_t* __restrict__ s, const Hdr& h, uint64_t b, BlockIn* out) {
  (void)h.g;
  const uint64_t gid = b / kGroup;
  const uint8_t* gp = s + h.L.groups + 24 * gid;
  unsigned long long pay = ld_u64(gp), un = ld_u64(gp + 8), rg = ld_u64(gp + 16);
  // sums over the group's blocks before b: eight 16-bit entries per 16-byte load (the
  // sections are 16-byte aligned and a group starts at a multiple of 256 entries), then the
  // partial last load; regression flags by whole bitmap words
  const uint64_t q0 = gid * kGroup, nq = b - q0;
  const uint4* sz4 = reinterpret_cast<const uint4*>(s + h.L.sizes + 2 * q0);
  const uint4* uc4 = reinterpret_cast<const uint4*>(s + h.L.ucounts + 2 * q0);
  auto sum16 = [](uint4 v, uint32_t n) {  // sum of the first n (<= 8) 16-bit entries
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t t = 0;
#pragma unroll
    for (uint32_t m = 0; m < 8; ++m)
      if (m < n) t += (w[m >> 1] >> (16 * (m & 1))) & 0xffffu;
    return t;
  };
  for (uint64_t q = 0; q < nq; q += 8) {
    const uint32_t n = (uint32_t)min((uint64_t)8, nq - q);
    pay += sum16(__ldg(sz4 + q / 8), n);
    un += sum16(__ldg(uc4 + q / 8), n);
  }
  const uint32_t* bm = reinterpret_cast<const uint32_t*>(s + h.L.bitmap) + q0 / 32;
  for (uint64_t q = 0; q < nq; q += 32) {
    const uint32_t n = (uint32_t)min((uint64_t)32, nq - q);
    const uint32_t word = __ldg(bm + q / 32);
    rg += __popc(n == 32 ? word : (word & ((1u << n) - 1)));
  }
  BlockIn& bi = *out;
  bi.b = b;
  bi.pay_off = pay;
  bi.un_off = un;
  bi.size = *reinterpret_cast<const uint16_t*>(s + h.L.sizes + 2 * b);
  bi.ucnt = *reinterpret_cast<const uint16_t*>(s + h.L.ucounts + 2 * b);
  const bool reg = (*reinterpret_cast<const uint32_t*>(s + h.L.bitmap + 4 * (b / 32)) >> (b % 32)) & 1u;
  bi.reg_idx = reg ? (int64_t)rg : -1;
  return !(pay + bi.size > h.payload_bytes || un + bi.ucnt > h.n_unpred || (reg && rg >= h.n_reg));
}

// Warp items of the fast decoder: item i is the 32 blocks [32 i, 32 i + 32), one per lane, all in
// group i / 8. The warp places them from the group's table entry and a warp scan of the group's
// block table (lane L sums entries 8L .. 8L+7, one 16-byte load each of the payload sizes and
// unpredictable counts; the regression flags by popcount of the group's 8 bitmap words), and
// checks the group's entry against the next one (as the CTA scan of a whole group does).
// Returns false, with a format error, when they disagree; then no block of the item is placed.
__device__ __forceinline__ bool warp_place(const uint8_t* __restrict__ s, const Hdr& h, uint64_t item,
                                           uint64_t ngroups, State* st, BlockIn* out) {
  const Geo& g = h.g;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t G = item >> 3, q0 = G * kGroup;
  const uint32_t m = (uint32_t)(item & 7);
  const uint32_t nblk = (uint32_t)min((uint64_t)kGroup, g.nb - q0);
  uint4 sz = make_uint4(0u, 0u, 0u, 0u), uc = sz;
  if (8 * lane < nblk) {
    sz = __ldg(reinterpret_cast<const uint4*>(s + h.L.sizes + 2 * q0) + lane);
    uc = __ldg(reinterpret_cast<const uint4*>(s + h.L.ucounts + 2 * q0) + lane);
  }
  const uint32_t lim = nblk > 8 * lane ? min(8u, nblk - 8 * lane) : 0u;  // entries of this lane's chunk in the group
  auto entry = [](const uint4& v, uint32_t e) {  // 16-bit entry e (< 8) of a chunk
    const uint32_t w = e < 2 ? v.x : (e < 4 ? v.y : (e < 6 ? v.z : v.w));
    return (w >> (16 * (e & 1))) & 0xffffu;
  };
  auto head = [&](const uint4& v, uint32_t n) {  // sum of the first n (<= 8) entries
    uint32_t t = 0;
#pragma unroll
    for (uint32_t e = 0; e < 8; ++e)
      if (e < n) t += entry(v, e);
    return t;
  };
  const uint32_t ssum = head(sz, lim), usum = head(uc, lim);
  uint32_t bw = 0;
  if (lane < 8 && 32 * lane < nblk) {
    bw = __ldg(reinterpret_cast<const uint32_t*>(s + h.L.bitmap) + q0 / 32 + lane);
    const uint32_t nb_w = nblk - 32 * lane;
    if (nb_w < 32) bw &= (1u << nb_w) - 1u;
  }
  uint32_t si = ssum, ui = usum, ri = __popc(bw);  // inclusive warp scans
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, si, o), b2 = __shfl_up_sync(0xffffffffu, ui, o),
                   c = __shfl_up_sync(0xffffffffu, ri, o);
    if (lane >= (uint32_t)o) {
      si += a;
      ui += b2;
      ri += c;
    }
  }
  const uint8_t* gp = s + h.L.groups + 24 * G;
  const unsigned long long base[3] = {ld_u64(gp), ld_u64(gp + 8), ld_u64(gp + 16)};
  const bool last = G + 1 >= ngroups;
  const unsigned long long next[3] = {last ? h.payload_bytes : ld_u64(gp + 24), last ? h.n_unpred : ld_u64(gp + 32),
                                      last ? h.n_reg : ld_u64(gp + 40)};
  const uint32_t tot_s = __shfl_sync(0xffffffffu, si, 31), tot_u = __shfl_sync(0xffffffffu, ui, 31),
                 tot_r = __shfl_sync(0xffffffffu, ri, 31);
  bool bad = base[0] + tot_s != next[0] || base[1] + tot_u != next[1] || base[2] + tot_r != next[2] ||
             (G == 0 && (base[0] | base[1] | base[2]) != 0);
  if (bad) {
    if (lane == 0) atomicOr(&st->error, ERR_FORMAT);
    return false;
  }
  // this lane's block: entry e = 32 m + lane of the group, in the chunk of lane e / 8
  const uint32_t e = 32 * m + lane, c = e >> 3, pos = e & 7;
  uint4 csz, cuc;
  csz.x = __shfl_sync(0xffffffffu, sz.x, c);
  csz.y = __shfl_sync(0xffffffffu, sz.y, c);
  csz.z = __shfl_sync(0xffffffffu, sz.z, c);
  csz.w = __shfl_sync(0xffffffffu, sz.w, c);
  cuc.x = __shfl_sync(0xffffffffu, uc.x, c);
  cuc.y = __shfl_sync(0xffffffffu, uc.y, c);
  cuc.z = __shfl_sync(0xffffffffu, uc.z, c);
  cuc.w = __shfl_sync(0xffffffffu, uc.w, c);
  const uint32_t sx = __shfl_sync(0xffffffffu, si - ssum, c), ux = __shfl_sync(0xffffffffu, ui - usum, c);
  const uint32_t word = __shfl_sync(0xffffffffu, bw, m), rx = __shfl_sync(0xffffffffu, ri - __popc(bw), m);
  BlockIn& bi = *out;
  bi.b = 32 * item + lane;
  bi.pay_off = base[0] + sx + head(csz, pos);
  bi.un_off = base[1] + ux + head(cuc, pos);
  bi.size = entry(csz, pos);
  bi.ucnt = entry(cuc, pos);
  const bool reg = (word >> lane) & 1u;
  const unsigned long long rg = base[2] + rx + __popc(word & ((1u << lane) - 1u));
  bi.reg_idx = reg ? (int64_t)rg : -1;
  return true;
}

__device__ __forceinline__ uint64_t warp_pull(unsigned long long* q) {
  unsigned long long v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(q, 1ull);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Generic kernel: edge blocks (or all blocks when `all`).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_decode(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h, T* field,
                                                uint8_t* status, const T* orig, State* st,
                                                const sdcsz_flip* __restrict__ flips, uint32_t nflips, int all) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Smem sm;
  uint32_t* lut = reinterpret_cast<uint32_t*>(smem);
  const uint16_t* syms = reinterpret_cast<const uint16_t*>(s + h.L.table + 4 * (kMaxLen + 1));
  if (!cta_tables(s, h, sm, lut, syms, st)) return;
  const Tables tb = {lut, &sm.cn, syms, h.n_live, nullptr};
  const uint8_t* lim = s + nbytes;
  Walker<T, NDIM> wk;
  wk.base = reinterpret_cast<T*>(smem + (4u << kLutBits)) + threadIdx.x;
  wk.stride = blockDim.x;
  wk.B2 = h.g.B[2];
  wk.sr = h.g.B[1] * h.g.B[2];
  const uint64_t ngroups = (h.g.nb + kGroup - 1) / kGroup;
  Acc acc;
  for (uint64_t gid = cta_pull(&st->queue[1]); gid < ngroups; gid = cta_pull(&st->queue[1])) {
    const uint64_t b0 = gid * kGroup;
    const uint32_t nblk = (uint32_t)min((uint64_t)kGroup, h.g.nb - b0);
    if (!all) {
      // skip groups without edge blocks
      int any = 0;
      for (uint32_t t = threadIdx.x; t < nblk; t += blockDim.x) any |= !is_full(h.g, b0 + t);
      if (!__syncthreads_or(any)) continue;
    }
    if (!group_scan(s, h, gid, ngroups, sm, st)) {
      if (status)
        for (uint32_t t = threadIdx.x; t < nblk; t += blockDim.x) status[b0 + t] = SDCSZ_BLOCK_BAD;
      continue;
    }
    for (uint32_t t = threadIdx.x; t < nblk; t += blockDim.x) {
      const uint64_t b = b0 + t;
      if (!all && is_full(h.g, b)) continue;
      BlockIn bi;
      bi.b = b;
      bi.pay_off = sm.off[t][0];
      bi.un_off = sm.off[t][1];
      bi.reg_idx = sm.rg[t] ? (int64_t)sm.off[t][2] : -1;
      bi.size = sm.sz[t];
      bi.ucnt = sm.uc[t];
      uint32_t kinj, bitinj;
      find_inj(flips, nflips, b, &kinj, &bitinj);
      const uint8_t stv = verify_block(s, h, b, [&](bool first, unsigned long long* sum, unsigned long long* nv,
                                                     double* me) {
        return decode_generic<T, NDIM>(s, lim, h, bi, tb, wk, FieldSink<T>{field}, orig, first ? kinj : kNone, bitinj, sum, nv, me);
      }, acc);
      if (status) status[b] = stv;
    }
  }
  acc.commit(st);
}

// Region decompression: the blocks that intersect a box, one thread each (enumerated over the
// box's block range), decoded and verified on their own (Sec. 5.1 random access) and stored
// into a dense array of the box's shape.
struct Region {
  uint64_t lo[3], hi[3];  // the box, padded 3D coordinates, [lo, hi)
  uint64_t c0[3], nc[3];  // its block range: first block coordinate and count per axis
};

template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_decode_region(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h, T* out,
                                                       Region rgn, uint8_t* status, State* st, uint64_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Smem sm;
  uint32_t* lut = reinterpret_cast<uint32_t*>(smem);
  const uint16_t* syms = reinterpret_cast<const uint16_t*>(s + h.L.table + 4 * (kMaxLen + 1));
  if (!cta_tables(s, h, sm, lut, syms, st)) return;
  const Tables tb = {lut, &sm.cn, syms, h.n_live, nullptr};
  const uint8_t* lim = s + nbytes;
  Walker<T, NDIM> wk;
  wk.base = reinterpret_cast<T*>(smem + (4u << kLutBits)) + threadIdx.x;
  wk.stride = blockDim.x;
  wk.B2 = h.g.B[2];
  wk.sr = h.g.B[1] * h.g.B[2];
  Acc acc;
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) {
    const Geo& g = h.g;
    const uint64_t r2 = e % rgn.nc[2], r = e / rgn.nc[2];
    const uint64_t r1 = r % rgn.nc[1], r0 = r / rgn.nc[1];
    const uint64_t b = ((rgn.c0[0] + r0) * g.nbd[1] + (rgn.c0[1] + r1)) * g.nbd[2] + (rgn.c0[2] + r2);
    RegionSink<T> sink;
    sink.out = out;
    for (int a = 0; a < 3; ++a) {
      sink.lo[a] = rgn.lo[a];
      sink.hi[a] = rgn.hi[a];
    }
    BlockIn bi;
    uint8_t stv;
    if (!place_block(s, h, b, &bi)) {
      atomicOr(&st->error, ERR_FORMAT);
      stv = SDCSZ_BLOCK_BAD;
      ++acc.bad;
    } else {
      stv = verify_block(s, h, b, [&](bool, unsigned long long* sum, unsigned long long* nv, double* me) {
        return decode_generic<T, NDIM>(s, lim, h, bi, tb, wk, sink, nullptr, kNone, 0, sum, nv, me);
      }, acc);
    }
    if (status) status[e] = stv;
  }
  acc.commit(st);
}

template <typename T, int NDIM, int B0, int B1, int B2, bool HOOK, bool WRITE, bool CMP>
__device__ __forceinline__ bool fast_dispatch(bool reg, const uint8_t* s, const uint8_t* lim, const Hdr& h,
                                              const BlockIn& bi, const Tables& tb, T* plane, T* out, const T* org,
                                              uint64_t si, uint64_t sj, bool vec2, uint32_t kinj, uint32_t bitinj,
                                              unsigned long long* sum, unsigned long long* nv, double* me) {
  if (reg)
    return decode_fast<T, NDIM, B0, B1, B2, true, HOOK, WRITE, CMP>(s, lim, h, bi, tb, plane, out, org, si, sj, vec2,
                                                                    kinj, bitinj, sum, nv, me);
  return decode_fast<T, NDIM, B0, B1, B2, false, HOOK, WRITE, CMP>(s, lim, h, bi, tb, plane, out, org, si, sj, vec2,
                                                                   kinj, bitinj, sum, nv, me);
}

// Fast kernel: full blocks of a compile-time shape (WRITE: decompression, else verification;
// CMP: compact encoding).
// The fast decoder's shared-memory tables (every thread of the CTA): the first-level table and
// the pair table in `smem`, the canonical tables in `sm`, and the pattern of a row of B2 central
// codes. False for a bad code table.
template <int B2, bool CMP>
__device__ __forceinline__ bool fast_tables(const uint8_t* s, const Hdr& h, Smem& sm, unsigned char* smem, State* st,
                                            Tables* tb) {
  uint32_t* lut = reinterpret_cast<uint32_t*>(smem);
  const uint16_t* syms = reinterpret_cast<const uint16_t*>(s + h.L.table + 4 * (kMaxLen + 1));
  __shared__ uint32_t s_central;  // central codeword: bits << 8 | length (0: none in the window)
  if (threadIdx.x == 0) s_central = 0;
  if (!cta_tables(s, h, sm, lut, syms, st)) return false;
  uint2* lut2 = reinterpret_cast<uint2*>(smem + (4u << kLutBits));
  __syncthreads();
  pair_table(lut2, lut, CMP);
  for (uint32_t e = threadIdx.x; e < (1u << kLutBits); e += blockDim.x) {  // every writer writes the same
    const uint32_t v = lut[e], l = v & 0xffu;
    if (l && (v >> 8) == h.g.R) s_central = ((e >> (kLutBits - l)) << 8) | l;
  }
  __syncthreads();
  uint32_t rbits = 0, rpat = 0;
  {
    const uint32_t lc = s_central & 0xffu, cc = s_central >> 8;
    if (lc && B2 * lc <= 32u) {
      rbits = B2 * lc;
#pragma unroll
      for (int l = 0; l < B2; ++l) rpat = (lc * (B2 - 1 - l) < 32u) ? (rpat | (cc << (lc * (B2 - 1 - l)))) : rpat;
    }
  }
  *tb = Tables{lut, &sm.cn, syms, h.n_live, lut2, rbits, rpat};
  return true;
}

// Edge blocks of a field whose full blocks take the fast kernel: one thread per edge block
// (compact enumeration), walked by the fast decoder's compile-time code at the block's extents;
// a block whose worst case could read past the stream takes the bounds-checked generic walk.
// Offsets from the stored group base plus the group's block table up to the block.
template <typename T, int NDIM, int B0, int B1, int B2, bool WRITE, bool CMP>
__global__ void __launch_bounds__(256, 2) k_decode_edges_fast(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h,
                                                              T* field, uint8_t* status, const T* orig, State* st,
                                                              const sdcsz_flip* __restrict__ flips, uint32_t nflips,
                                                              uint64_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Smem sm;
  Tables tb;
  if (!fast_tables<B2, CMP>(s, h, sm, smem, st, &tb)) return;
  const uint8_t* lim = s + nbytes;
  T* plane = reinterpret_cast<T*>(smem + (12u << kLutBits)) + threadIdx.x;
  Walker<T, NDIM> wk;
  wk.base = plane;
  wk.stride = blockDim.x;
  wk.B2 = B2;
  wk.sr = B1 * B2;
  const Geo& g = h.g;
  const uint64_t si = g.d[1] * g.d[2], sj = g.d[2];
  Acc acc;
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) {
    const uint64_t b = edge_block(g, e);
    const Box x = block_box(g, b);
    BlockIn bi;
    uint8_t stv;
    if (!place_block(s, h, b, &bi)) {
      atomicOr(&st->error, ERR_FORMAT);
      stv = SDCSZ_BLOCK_BAD;
      ++acc.bad;
    } else {
      const uint64_t bo = row_base(g, x, 0, 0);
      T* out = WRITE ? field + bo : nullptr;
      const T* org = (!WRITE && orig) ? orig + bo : nullptr;
      const bool reg = bi.reg_idx >= 0;
      uint32_t kinj, bitinj;
      find_inj(flips, nflips, b, &kinj, &bitinj);
      const uint64_t worst = CMP ? (3ull + sizeof(T)) * (B0 * B1 * B2) + 19 : 3ull * (B0 * B1 * B2);
      const bool safe = (uint64_t)(lim - (s + h.L.payload)) >= bi.pay_off + worst + 16;
      stv = verify_block(s, h, b, [&](bool first, unsigned long long* sum, unsigned long long* nv, double* me) {
        if (!safe)
          return decode_generic<T, NDIM>(s, lim, h, bi, tb, wk, FieldSink<T>{field}, orig, first ? kinj : kNone,
                                         bitinj, sum, nv, me);
        const uint32_t ki = first ? kinj : kNone;
        if (reg) {
          if (ki != kNone)
            return decode_fast<T, NDIM, B0, B1, B2, true, true, WRITE, CMP, true>(
                s, lim, h, bi, tb, plane, out, org, si, sj, false, ki, bitinj, sum, nv, me, x.e[0], x.e[1], x.e[2]);
          return decode_fast<T, NDIM, B0, B1, B2, true, false, WRITE, CMP, true>(
              s, lim, h, bi, tb, plane, out, org, si, sj, false, kNone, 0, sum, nv, me, x.e[0], x.e[1], x.e[2]);
        }
        if (ki != kNone)
          return decode_fast<T, NDIM, B0, B1, B2, false, true, WRITE, CMP, true>(
              s, lim, h, bi, tb, plane, out, org, si, sj, false, ki, bitinj, sum, nv, me, x.e[0], x.e[1], x.e[2]);
        return decode_fast<T, NDIM, B0, B1, B2, false, false, WRITE, CMP, true>(
            s, lim, h, bi, tb, plane, out, org, si, sj, false, kNone, 0, sum, nv, me, x.e[0], x.e[1], x.e[2]);
      }, acc);
    }
    if (status) status[b] = stv;
  }
  acc.commit(st);
}

template <typename T, int NDIM, int B0, int B1, int B2, bool WRITE, bool CMP>
__device__ __forceinline__ void decode_fast_cta(const uint8_t* __restrict__ s, uint64_t nbytes, const Hdr& h, T* field,
                                                uint8_t* status, const T* orig, State* st,
                                                const sdcsz_flip* __restrict__ flips, uint32_t nflips, int vec2,
                                                unsigned char* smem) {
  __shared__ Smem sm;
  Tables tb;
  if (!fast_tables<B2, CMP>(s, h, sm, smem, st, &tb)) return;
  const uint8_t* lim = s + nbytes;
  T* plane = reinterpret_cast<T*>(smem + (12u << kLutBits)) + threadIdx.x;
  Walker<T, NDIM> wk;  // for the few blocks that take the generic decoder
  wk.base = plane;
  wk.stride = blockDim.x;
  wk.B2 = B2;
  wk.sr = B1 * B2;
  const Geo& g = h.g;
  const uint64_t si = g.d[1] * g.d[2], sj = g.d[2];
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  Acc acc;
  // warp items (32 blocks) from the queue, one ahead: the next item's block-table lines are on
  // their way to L2 while this one is decoded; no barrier between the CTA's warps
  const uint64_t nitems = (g.nb + 31) / 32;
  const uint32_t lane = threadIdx.x & 31;
  // Items are placed one ahead: while item i is decoded, item i+1's blocks are already placed and
  // the head of each one's payload, its coefficients and its sum_dc are on their way to L2.
  auto prefetch_block = [&](const BlockIn& q, uint64_t it) {
    if (32 * it + lane >= g.nb) return;
    const uint64_t offs[3] = {h.L.payload + q.pay_off, h.L.coef + (q.reg_idx >= 0 ? (uint64_t)q.reg_idx : 0ull) *
                                                                         (uint64_t)(NDIM + 1) * sizeof(T),
                              h.L.sumdc + 8 * (32 * it + lane)};
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if ((k != 1 || (q.reg_idx >= 0 && !CMP)) && (k != 2 || g.abft) && offs[k] < nbytes) prefetch_l2(s + offs[k]);
  };
  // the block-table, unpredictable-count and group-table lines of an item, two items ahead
  auto prefetch_tables = [&](uint64_t it) {  // what warp_place reads: the whole group's tables
    if (it >= nitems || lane >= 11) return;
    const uint64_t G = it >> 3;
    uint64_t off;
    if (lane < 4) off = h.L.sizes + 512 * G + 128 * lane;
    else if (lane < 8) off = h.L.ucounts + 512 * G + 128 * (lane - 4);
    else if (lane == 8) off = h.L.bitmap + 32 * G;
    else off = h.L.groups + 24 * G + 24 * (lane - 9);  // this group's entry and the next one's
    if (off < nbytes) prefetch_l2(s + off);
  };
  uint64_t item = warp_pull(&st->queue[0]);
  BlockIn bi;
  bool placed = item < nitems && warp_place(s, h, item, ngroups, st, &bi);
  uint64_t nxt = warp_pull(&st->queue[0]);
  prefetch_tables(nxt);
  while (item < nitems) {
    const uint64_t nn = warp_pull(&st->queue[0]);
    prefetch_tables(nn);
    BlockIn bn;
    const bool placed_n = nxt < nitems && warp_place(s, h, nxt, ngroups, st, &bn);
    if (placed_n) prefetch_block(bn, nxt);
    const uint64_t b = 32 * item + lane;
    if (!placed) {
      if (status && b < g.nb) status[b] = SDCSZ_BLOCK_BAD;
      item = nxt;
      nxt = nn;
      bi = bn;
      placed = placed_n;
      continue;
    }
    bool full = false;
    uint64_t bo = 0;
    if (b < g.nb) {
      uint64_t c0, c1, c2;
      block_coords(g, b, c0, c1, c2);
      full = (c0 + 1) * B0 <= g.d[0] && (c1 + 1) * B1 <= g.d[1] && (c2 + 1) * B2 <= g.d[2];
      bo = (c0 * B0 * g.d[1] + c1 * B1) * g.d[2] + c2 * B2;
    }
    if (full) {
      T* out = WRITE ? field + bo : nullptr;
      const T* org = (!WRITE && orig) ? orig + bo : nullptr;
      const bool reg = bi.reg_idx >= 0;
      uint32_t kinj, bitinj;
      find_inj(flips, nflips, b, &kinj, &bitinj);
      // The unchecked reader consumes at most 24 bits per point whatever the data (in the compact
      // encoding also a whole value per point and 4 coefficients of at most 38 bits), reads at
      // most 12 bytes ahead of what it consumed and starts up to 3 bytes early; blocks whose
      // worst case could reach the end of the stream take the bounds-checked reader.
      const uint64_t worst = CMP ? (3ull + sizeof(T)) * (B0 * B1 * B2) + 19 : 3ull * (B0 * B1 * B2);
      const bool safe = (uint64_t)(lim - (s + h.L.payload)) >= bi.pay_off + worst + 16;
      const bool in_range = !(bi.pay_off + bi.size > h.payload_bytes || bi.un_off + bi.ucnt > h.n_unpred ||
                              (reg && (uint64_t)bi.reg_idx >= h.n_reg));
      uint8_t stv = SDCSZ_BLOCK_BAD;
      if (in_range)
        stv = verify_block(s, h, b, [&](bool first, unsigned long long* sum, unsigned long long* nv, double* me) {
          if (!safe)
            return decode_generic<T, NDIM>(s, lim, h, bi, tb, wk, FieldSink<T>{field}, orig, first ? kinj : kNone,
                                           bitinj, sum, nv, me);
          if (first && kinj != kNone)
            return fast_dispatch<T, NDIM, B0, B1, B2, true, WRITE, CMP>(reg, s, lim, h, bi, tb, plane, out, org, si, sj,
                                                                        vec2, kinj, bitinj, sum, nv, me);
          return fast_dispatch<T, NDIM, B0, B1, B2, false, WRITE, CMP>(reg, s, lim, h, bi, tb, plane, out, org, si,
                                                                       sj, vec2, kNone, 0, sum, nv, me);
        }, acc);
      else
        ++acc.bad;
      if (status) status[b] = stv;
    }
    item = nxt;
    nxt = nn;
    bi = bn;
    placed = placed_n;
  }
  acc.commit(st);
}

// The raw and compact kernels, held to two CTAs per SM (128 registers): left to itself the
// compiler spills some variants at 80 registers.
template <typename T, int NDIM, int B0, int B1, int B2, bool WRITE>
__global__ void __launch_bounds__(256, 2) k_decode_fast(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h, T* field,
                                                     uint8_t* status, const T* orig, State* st,
                                                     const sdcsz_flip* __restrict__ flips, uint32_t nflips,
                                                     int vec2) {
  extern __shared__ __align__(16) unsigned char smem[];
  decode_fast_cta<T, NDIM, B0, B1, B2, WRITE, false>(s, nbytes, h, field, status, orig, st, flips, nflips, vec2, smem);
}

template <typename T, int NDIM, int B0, int B1, int B2, bool WRITE>
__global__ void __launch_bounds__(256, 2) k_decode_fast_c(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h,
                                                          T* field, uint8_t* status, const T* orig, State* st,
                                                          const sdcsz_flip* __restrict__ flips, uint32_t nflips,
                                                          int vec2) {
  extern __shared__ __align__(16) unsigned char smem[];
  decode_fast_cta<T, NDIM, B0, B1, B2, WRITE, true>(s, nbytes, h, field, status, orig, st, flips, nflips, vec2, smem);
}

// ---------------------------------------------------------------- launch
template <class K>
inline unsigned persistent_grid(K kern, uint32_t threads, size_t smem, uint64_t ngroups, const Launch& L) {
  const int occ = occupancy(reinterpret_cast<const void*>(kern), (int)threads, smem);
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ngroups, (uint64_t)occ * L.sms));
}

// CMP: the compact encoding's kernels (instantiated in their own translation units).
template <typename T, int NDIM, int B0, int B1, int B2, bool CMP>
void run_fast(const uint8_t* s, uint64_t nbytes, const Hdr& h, T* field, uint8_t* status, const T* orig, State* st,
              const sdcsz_flip* flips, uint32_t nflips, const Launch& L, const Launch& Le) {
  const size_t smem = (12u << kLutBits) + (size_t)walker_slots(NDIM, h.g.B) * 256 * sizeof(T);  // lut, pair lut, plane
  // the edge blocks, on Le (the side stream), with the same compile-time walk at their extents
  if (const uint64_t count = edge_count(h.g)) {
    auto ke = field ? k_decode_edges_fast<T, NDIM, B0, B1, B2, true, CMP>
                    : k_decode_edges_fast<T, NDIM, B0, B1, B2, false, CMP>;
    allow_smem(reinterpret_cast<const void*>(ke), smem);
    ke<<<(unsigned)((count + 255) / 256), 256, smem, Le.stream>>>(s, nbytes, h, field, status, orig, st, flips, nflips,
                                                                   count);
    note_launch();
  }
  auto kern = CMP ? (field ? k_decode_fast_c<T, NDIM, B0, B1, B2, true> : k_decode_fast_c<T, NDIM, B0, B1, B2, false>)
                  : (field ? k_decode_fast<T, NDIM, B0, B1, B2, true> : k_decode_fast<T, NDIM, B0, B1, B2, false>);
  const uint64_t ngroups = (h.g.nb + kGroup - 1) / kGroup;
  const unsigned grid = persistent_grid(kern, 256, smem, ngroups, L);
  const uintptr_t al = 2 * sizeof(T);
  const bool vec2 = (B2 % 2 == 0) && (h.g.d[2] % 2 == 0) && (reinterpret_cast<uintptr_t>(field) % al == 0);
  kern<<<grid, 256, smem, L.stream>>>(s, nbytes, h, field, status, orig, st, flips, nflips, vec2 ? 1 : 0);
  note_launch();
}

template <typename T>
bool has_fast(const Geo& g) {
  if (g.ndim == 3 && g.B[0] == g.B[1] && g.B[1] == g.B[2])
    return g.B[2] == 4 || g.B[2] == 6 || g.B[2] == 8 || (sizeof(T) == 4 && (g.B[2] == 10 || g.B[2] == 12));
  if (g.ndim == 2 && g.B[1] == g.B[2]) return g.B[2] == 8 || g.B[2] == 12 || g.B[2] == 16;
  return false;
}

template <typename T, bool CMP>
bool try_fast(const uint8_t* s, uint64_t nbytes, const Hdr& h, T* field, uint8_t* status, const T* orig, State* st,
              const sdcsz_flip* flips, uint32_t nflips, const Launch& L, const Launch& Le) {
  const Geo& g = h.g;
  // a 3D 16^3 float64 plane would not fit 256 threads' shared memory: generic path
  if (g.ndim == 3 && g.B[0] == g.B[1] && g.B[1] == g.B[2]) {
    switch (g.B[2]) {
      case 4: run_fast<T, 3, 4, 4, 4, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le); return true;
      case 6: run_fast<T, 3, 6, 6, 6, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le); return true;
      case 8: run_fast<T, 3, 8, 8, 8, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le); return true;
      case 10:
        if (sizeof(T) == 8) return false;
        run_fast<T, 3, 10, 10, 10, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le);
        return true;
      case 12:
        if (sizeof(T) == 8) return false;
        run_fast<T, 3, 12, 12, 12, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le);
        return true;
      default: return false;
    }
  }
  if (g.ndim == 2 && g.B[1] == g.B[2]) {
    switch (g.B[2]) {
      case 8: run_fast<T, 2, 1, 8, 8, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le); return true;
      case 12: run_fast<T, 2, 1, 12, 12, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le); return true;
      case 16: run_fast<T, 2, 1, 16, 16, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, Le); return true;
      default: return false;
    }
  }
  return false;
}

template <typename T, int NDIM>
void run_generic(const uint8_t* s, uint64_t nbytes, const Hdr& h, T* field, uint8_t* status, const T* orig, State* st,
                 const sdcsz_flip* flips, uint32_t nflips, bool all, const Launch& L) {
  const size_t per = (size_t)walker_slots(h.g.ndim, h.g.B) * sizeof(T);
  uint32_t threads = 256;
  while (threads > 64 && per * threads > 192 * 1024) threads >>= 1;
  const size_t smem = (4u << kLutBits) + per * threads;
  auto kern = k_decode<T, NDIM>;
  const uint64_t ngroups = (h.g.nb + kGroup - 1) / kGroup;
  const unsigned grid = persistent_grid(kern, threads, smem, ngroups, L);
  kern<<<grid, threads, smem, L.stream>>>(s, nbytes, h, field, status, orig, st, flips, nflips, all ? 1 : 0);
  note_launch();
}

// Fields whose block shape has a fast path: full blocks on the caller's stream, edge blocks on the
// side stream (the encoding fixed at compile time).
template <typename T, bool CMP>
void launch_decode_fast_t(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field_v, uint8_t* status,
                          const void* orig_v, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                          const Launch& L) {
  if (h.g.nb == 0) return;
  T* field = write ? static_cast<T*>(field_v) : nullptr;
  const T* orig = static_cast<const T*>(orig_v);
  Fork fk(L);
  try_fast<T, CMP>(s, nbytes, h, field, status, orig, st, flips, nflips, L, fk.side_launch(L));
  fk.join();
}

// Other shapes: the generic kernel for every block (either encoding).
template <typename T>
void launch_decode_generic_t(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field_v, uint8_t* status,
                             const void* orig_v, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                             const Launch& L) {
  if (h.g.nb == 0) return;
  T* field = write ? static_cast<T*>(field_v) : nullptr;
  const T* orig = static_cast<const T*>(orig_v);
  if (h.g.ndim == 3) run_generic<T, 3>(s, nbytes, h, field, status, orig, st, flips, nflips, true, L);
  else if (h.g.ndim == 2) run_generic<T, 2>(s, nbytes, h, field, status, orig, st, flips, nflips, true, L);
  else run_generic<T, 1>(s, nbytes, h, field, status, orig, st, flips, nflips, true, L);
}

template <typename T>
void launch_region_t(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* out, const Region& rgn, uint8_t* status,
                     State* st, const Launch& L) {
  const uint64_t count = rgn.nc[0] * rgn.nc[1] * rgn.nc[2];
  if (!count) return;
  const size_t per = (size_t)walker_slots(h.g.ndim, h.g.B) * sizeof(T);
  uint32_t threads = 256;
  while (threads > 64 && per * threads > 192 * 1024) threads >>= 1;
  const size_t smem = (4u << kLutBits) + per * threads;
  const unsigned grid = (unsigned)((count + threads - 1) / threads);
  T* o = static_cast<T*>(out);
  if (h.g.ndim == 3) {
    allow_smem(reinterpret_cast<const void*>(k_decode_region<T, 3>), smem);
    k_decode_region<T, 3><<<grid, threads, smem, L.stream>>>(s, nbytes, h, o, rgn, status, st, count);
  } else if (h.g.ndim == 2) {
    allow_smem(reinterpret_cast<const void*>(k_decode_region<T, 2>), smem);
    k_decode_region<T, 2><<<grid, threads, smem, L.stream>>>(s, nbytes, h, o, rgn, status, st, count);
  } else {
    allow_smem(reinterpret_cast<const void*>(k_decode_region<T, 1>), smem);
    k_decode_region<T, 1><<<grid, threads, smem, L.stream>>>(s, nbytes, h, o, rgn, status, st, count);
  }
  note_launch();
}

}  // namespace
}  // namespace kdec
}  // namespace sdcsz
