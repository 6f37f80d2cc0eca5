// K4: per-block Huffman encoding and stream assembly (the encoding and output steps of
// Algorithm 1 of the paper, without the Zstd stage). Two kernels:
//
// K4a, one thread per block: encodes the block's codes (read from HBM once) MSB-first into a
// fixed-size slot of the workspace, taking sum_q/isum_q on the way. In the compact encoding
// the block's coefficient integers come first and each unpredictable value follows its code
// 0, truncated to the mantissa bits the bound needs. When they disagree with
// the values of K2 (Algorithm 1's check of the bin array before encoding) the single corrupted
// code is located and repaired and the block is encoded again. Then the block's unpredictable
// values move to the front of its staging slot, and the per-block entries that sit at fixed
// places in the stream (payload size, unpredictable count, sum_dc, regression bitmap) are
// written; each warp adds its 32 blocks' payload bytes, unpredictables and regression blocks
// to its group's totals (one 64-bit atomic).
//
// K4b, one CTA per random-access group of 256 blocks: a CTA scan plus the sum of the earlier
// groups' totals (no CTA waits on another) gives each block its payload, unpredictable-value
// and coefficient offsets; each thread then copies
// its block's payload (the slot holds it in stream byte order: whole aligned words are stored
// with a funnel shift, the partial first and last words byte by byte), its unpredictable values
// and its coefficients. The group's table entry and, for the last group, the header totals are
// written.
#include <algorithm>

#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

// totals of a group (group_total_words): bytes (25 bits: 256 blocks of at most 65535), unpredictable
// points (21 bits: 256 blocks of at most 4096), regression blocks (16 bits)
constexpr unsigned long long kMaskBytes = (1ull << 25) - 1, kMaskUn = (1ull << 21) - 1;
constexpr uint32_t kCbWindow = 2048;  // codebook entries around the centre kept in shared memory
constexpr uint32_t kPosKept = 4;      // unpredictable positions remembered in registers per block

__device__ __forceinline__ unsigned long long pack_tot(unsigned long long bytes, unsigned long long un,
                                                       unsigned long long rg) {
  return (rg << 46) | (un << 25) | bytes;
}

__device__ __forceinline__ void mad_wide(unsigned long long& acc, uint32_t a, uint32_t b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

struct Codebook {
  const uint32_t* s;  // shared window [lo, lo + kCbWindow)
  const uint32_t* g;
  uint32_t lo;
  __device__ __forceinline__ uint32_t operator()(uint32_t c) const {
    const uint32_t d = c - lo;
    return d < kCbWindow ? s[d] : __ldg(&g[c]);
  }
};

__device__ __forceinline__ uint32_t cb_lo(const Geo& g) { return g.R > kCbWindow / 2 ? g.R - kCbWindow / 2 : 0; }

// Shared-memory window of the codebook around the centre bin.
__device__ __forceinline__ void cb_load(uint32_t* cb_s, const Geo& g, const Ws& w) {
  const uint32_t lo = cb_lo(g);
  for (uint32_t q = threadIdx.x; q < kCbWindow; q += blockDim.x)
    cb_s[q] = lo + q < g.bins ? __ldg(&w.codebook[lo + q]) : 0u;
}

// The error flag read once by the CTA, so that every thread takes the same path.
__device__ __forceinline__ bool cta_failed(State* st) {
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = *(volatile unsigned int*)&st->error != 0;
  __syncthreads();
  return s_fail != 0;
}

struct EncRes {
  uint32_t bits, nun, sq;
  unsigned long long isq;
  uint32_t pos[kPosKept];
};

// What the compact encoding adds to a block's payload: its coefficient integers (nco of
// them, none for a Lorenzo block) and, after each code 0, the point's value from the
// unpredictable staging (stride 32) truncated at exponent texp.
template <typename T>
struct Extra {
  const int* kq;
  int nco;
  const T* up;
  int texp;
};

// Code pairs reach the encoder through a ring of kRing batches of 8 pair rows in shared memory
// (word q of slot r of thread t at ((r * 8 + q) * kRingStride + t)), filled by cp.async while
// kRing - 1 batches are in flight: a warp's 32 blocks keep each pair row in one 128-byte line
// (the pairs are warp-interleaved), so the warp copies 8 rows with two 16-byte copies per lane
// and shares them after a warp barrier. Every lane of the warp runs the ring over the pairs the
// layout keeps per block, whatever its own block's size.
constexpr uint32_t kRing = 3;
constexpr uint32_t kRingStride = 128;  // threads of the encoding kernels' CTAs

__device__ __forceinline__ void cp_async4(uint32_t* dst_smem, const uint32_t* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t* dst_smem, const uint32_t* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One pass over a block's codes: the Huffman bits into `slot` (stream byte order, the last
// word zero padded), the code checksums (ABFT), the unpredictable count and the first
// kPosKept unpredictable positions. With FIX, code kfix reads as vfix. CMP: compact encoding.
// R is the central code (prediction within half a bin). pa: the pairs the staging layout keeps
// per block (pairs_of of the full block). ring: this thread's staging ring (nullptr: the pairs
// are loaded from memory directly).
template <bool ABFT, bool FIX, bool CMP, typename T>
__device__ __forceinline__ EncRes encode_codes(const uint32_t* __restrict__ pp, uint32_t P, uint32_t* __restrict__ slot,
                                               const Codebook& cb, uint32_t cw0, uint32_t R, uint32_t kfix,
                                               uint32_t vfix, const Extra<T>& ex, uint32_t pa,
                                               uint32_t* ring = nullptr) {
  EncRes e;
  e.bits = 0;
  e.nun = 0;
  e.sq = 0;
  e.isq = 0;
  unsigned long long acc = 0;
  uint32_t nacc = 0, wi = 0;
  // len (<= 32) low bits of v
  auto put_bits = [&](uint32_t v, uint32_t len) {
    acc = (acc << len) | (len < 32 ? (v & ((1u << len) - 1u)) : v);
    nacc += len;
    e.bits += len;
    if (nacc >= 32) {
      nacc -= 32;
      slot[wi++] = __byte_perm((uint32_t)(acc >> nacc), 0, 0x0123);
    }
  };
  auto put_value = [&](uint32_t k) {
    typedef typename Bitsof<T>::U U;
    const T v = ex.up[32 * (uint64_t)k];
    const int m = kept_bits<T>(v, ex.texp);
    const uint32_t len = 1u + Bitsof<T>::E + (uint32_t)m;
    const U u = Bitsof<T>::raw(v) >> (Bitsof<T>::M - m);
    if (len > 32) put_bits((uint32_t)((unsigned long long)u >> 32), len - 32);
    put_bits((uint32_t)u, len > 32 ? 32u : len);
  };
  if (CMP)
    for (int a = 0; a < ex.nco; ++a) {  // zigzag, its bit length in 6 bits, the bits below the leading one
      const int kv = ex.kq[a];
      const uint32_t z = ((uint32_t)kv << 1) ^ (kv < 0 ? 0xffffffffu : 0u);
      const uint32_t n = 32u - (uint32_t)__clz(z);
      put_bits(n, 6);
      if (n > 1) put_bits(z, n - 1);
    }
  auto put = [&](uint32_t c, uint32_t k) {
    if (FIX && k == kfix) c = vfix;
    const uint32_t cw = c ? cb(c) : cw0;
    const uint32_t len = cw & 31u;
    acc = (acc << len) | (cw >> 5);
    nacc += len;
    e.bits += len;
    if (nacc >= 32) {
      nacc -= 32;
      slot[wi++] = __byte_perm((uint32_t)(acc >> nacc), 0, 0x0123);
    }
    if (ABFT) {
      e.sq += c;
      mad_wide(e.isq, c, k + 1);
    }
    if (c == 0) {
      if (e.nun < kPosKept) e.pos[e.nun] = k;
      ++e.nun;
      if (CMP) put_value(k);
    }
  };
  // Both codes of a pair at once when their bits fit in one word (nearly always: codes are a
  // few bits long); the accumulator then holds at most 31 + 32 bits before its one flush.
  auto put2 = [&](uint32_t c0, uint32_t c1, uint32_t k) {
    if (FIX && k == kfix) c0 = vfix;
    if (FIX && k + 1 == kfix) c1 = vfix;
    const uint32_t w0 = c0 ? cb(c0) : cw0, w1 = c1 ? cb(c1) : cw0;
    const uint32_t l0 = w0 & 31u, l1 = w1 & 31u, l = l0 + l1;
    if (l > 32 || (CMP && (c0 == 0 || c1 == 0))) {
      put(c0, k);
      put(c1, k + 1);
      return;
    }
    acc = (acc << l) | (((unsigned long long)(w0 >> 5) << l1) | (w1 >> 5));
    nacc += l;
    e.bits += l;
    if (nacc >= 32) {
      nacc -= 32;
      slot[wi++] = __byte_perm((uint32_t)(acc >> nacc), 0, 0x0123);
    }
    if (ABFT) {
      e.sq += c0 + c1;
      mad_wide(e.isq, c0 + c1, k + 1);  // (k+1) c0 + (k+2) c1
      e.isq += c1;
    }
    if (c0 == 0 || c1 == 0) {
      if (c0 == 0) {
        if (e.nun < kPosKept) e.pos[e.nun] = k;
        ++e.nun;
      }
      if (c1 == 0) {
        if (e.nun < kPosKept) e.pos[e.nun] = k + 1;
        ++e.nun;
      }
    }
  };
  // Eight central codes in a row (the common case of a smooth field) go in with one append of
  // the central codeword repeated eight times, their checksums in closed form: sum_q gains 8 R
  // and isum_q gains R (8k + 36) for codes k .. k+7. The bits are those of eight single appends
  // (one flush suffices: fewer than 32 bits were pending and the run adds at most 32). With a
  // central codeword of at most 2 bits, sixteen at once the same way (R (16k + 136)).
  const uint32_t cwc = cb(R), lc = cwc & 31u, lrun = 8 * lc;
  const bool runs = !FIX && lc != 0 && lc <= 4;
  const bool runs16 = runs && lc <= 2;
  uint32_t rep = 0;
  if (runs)
#pragma unroll
    for (int t = 0; t < 8; ++t) rep = (rep << lc) | (cwc >> 5);
  const uint32_t rep16 = runs16 ? ((rep << lrun) | rep) : 0u;
  const uint32_t pc = R | (R << 16);  // a pair word of two central codes
  // code pairs eight at a time, the next eight loaded while these are encoded
  const uint32_t P2 = P >> 1;
  uint32_t wq[8], wn[8];
  auto load8 = [&](uint32_t base, uint32_t (&w)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) w[q] = (base + q < P2) ? pp[32 * (uint64_t)(base + q)] : 0u;
  };
  // batch `base` into ring slot `sl`: every pair below pa (the pairs the layout keeps per
  // block) lies inside the staging array, so only a batch reaching past pa needs a test
  const uint32_t lane = threadIdx.x & 31;
  auto stage8 = [&](uint32_t base, uint32_t sl) {
    // lane L: 16 bytes (lanes 4c .. 4c+3, c = L mod 8) of rows base + L/8 and base + 4 + L/8
    const uint32_t c = 4 * (lane & 7), q0 = lane >> 3;
    uint32_t* r = ring - lane + sl * 8 * kRingStride + c;
    const uint32_t* src = pp - lane + 32 * (uint64_t)base + c;
#pragma unroll
    for (uint32_t q = q0; q < 8; q += 4)
      if (base + q < pa) cp_async16(r + q * kRingStride, src + 32 * q);
    cp_async_commit();
  };
  uint32_t s_in = kRing - 1, s_out = 0;  // ring slots of the next batch staged and consumed
  if (ring) {
#pragma unroll
    for (uint32_t t = 0; t < kRing - 1; ++t) stage8(8 * t, t);
  } else {
    load8(0, wq);
  }
  const uint32_t nk = ring ? pa : P2;  // the ring's loop is the same for the whole warp
  for (uint32_t k8 = 0; k8 < nk; k8 += 8) {
    if (ring) {
      __syncwarp();  // every lane is done with the slot the next batch goes to
      stage8(k8 + 8 * (kRing - 1), s_in);  // an empty group past the end keeps the count uniform
      s_in = s_in + 1 == kRing ? 0 : s_in + 1;
      cp_async_wait<kRing - 1>();
      __syncwarp();  // the other lanes' copies of this batch are visible
      const uint32_t* r = ring + s_out * 8 * kRingStride;
      s_out = s_out + 1 == kRing ? 0 : s_out + 1;
#pragma unroll
      for (int q = 0; q < 8; ++q) wq[q] = r[q * kRingStride];
    } else if (k8 + 8 < P2) {
      load8(k8 + 8, wn);
    }
    if (runs16 && k8 + 8 <= P2 &&
        (((wq[0] ^ pc) | (wq[1] ^ pc) | (wq[2] ^ pc) | (wq[3] ^ pc)) |
         ((wq[4] ^ pc) | (wq[5] ^ pc) | (wq[6] ^ pc) | (wq[7] ^ pc))) == 0u) {
      acc = (acc << (2 * lrun)) | rep16;
      nacc += 2 * lrun;
      e.bits += 2 * lrun;
      if (nacc >= 32) {
        nacc -= 32;
        slot[wi++] = __byte_perm((uint32_t)(acc >> nacc), 0, 0x0123);
      }
      if (ABFT) {
        e.sq += 16 * R;
        mad_wide(e.isq, R, 32 * k8 + 136);  // codes k = 2 k8 .. k + 15: 16 k + 136
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k2 = k8 + 4 * h;
        if (runs && k2 + 3 < P2 &&
            ((wq[4 * h] ^ pc) | (wq[4 * h + 1] ^ pc) | (wq[4 * h + 2] ^ pc) | (wq[4 * h + 3] ^ pc)) == 0u) {
          acc = (acc << lrun) | rep;
          nacc += lrun;
          e.bits += lrun;
          if (nacc >= 32) {
            nacc -= 32;
            slot[wi++] = __byte_perm((uint32_t)(acc >> nacc), 0, 0x0123);
          }
          if (ABFT) {
            e.sq += 8 * R;
            mad_wide(e.isq, R, 16 * k2 + 36);  // codes k = 2 k2 .. k + 7: 8 k + 36
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (k2 + q < P2) put2(wq[4 * h + q] & 0xffffu, wq[4 * h + q] >> 16, 2 * (k2 + q));
        }
      }
    }
    if (!ring) {
#pragma unroll
      for (int q = 0; q < 8; ++q) wq[q] = wn[q];
    }
  }
  if (ring) cp_async_wait<0>();
  if (P & 1) put(pp[32 * (uint64_t)P2] & 0xffffu, P - 1);
  if (nacc) slot[wi] = __byte_perm((uint32_t)(acc << (32 - nacc)), 0, 0x0123);
  return e;
}

// Store the little-endian word `v` at aligned word address `wa` of the stream, keeping only
// the bytes inside [lo, hi).
__device__ __forceinline__ void put_bytes(uint8_t* out, uint64_t wa, uint32_t v, uint64_t lo, uint64_t hi) {
  for (int q = 0; q < 4; ++q)
    if (wa + q >= lo && wa + q < hi) out[wa + q] = (uint8_t)(v >> (8 * q));
}

// Payload slot of one block, 16-byte rounded: P codes of at most kMaxLen bits; in the compact
// encoding also a whole value per point and 4 coefficient integers of at most 38 bits.
__host__ __device__ inline uint64_t slot_words_of(const Geo& g) {
  const uint64_t bits = (uint64_t)g.P * (kMaxLen + (g.enc ? 8 * (g.dtype ? 8 : 4) : 0)) + (g.enc ? 4 * 38 : 0);
  return (bits + 127) / 128 * 4;
}

// ---------------------------------------------------------------- K4a
// field (nullable): the input, for the values of points whose codes an uncorrectable corruption
// turned into code 0 (K2 staged values only for the points it found unpredictable).
template <typename T, bool ABFT, bool CMP>
__device__ __forceinline__ void encode_block(const Geo& g, const Ws& w, uint8_t* __restrict__ out,
                                             const uint32_t* cb_s, uint64_t b, uint32_t* ring,
                                             const Shard& sh = Shard{}, const T* __restrict__ field = nullptr) {
  State* st = w.st;
  const Layout L = st->L;
  const uint32_t lane = threadIdx.x & 31;
  const bool active = b < g.nb;
  bool reg = false;
  unsigned long long nun_enc = 0;
  uint32_t nbytes = 0;
  // the first pass stages the warp's codes together (ring): every lane of the warp takes part,
  // and a lane past the field's blocks encodes nothing (P = 0)
  Codebook cb;
  cb.lo = cb_lo(g);
  cb.s = cb_s;
  cb.g = w.codebook;
  const uint32_t cw0 = __ldg(&w.codebook[0]);
  const uint32_t P = active ? block_box(g, b).P : 0u;
  reg = active && (w.flags[b] & 1);
  // what the checks after the encoding compare and copy, loaded now (in flight meanwhile)
  const unsigned long long sq_ref = (ABFT && active) ? w.sum_q[b] : 0ull;
  const unsigned long long isq_ref = (ABFT && active) ? w.isum_q[b] : 0ull;
  const unsigned long long sdc_ref = (ABFT && active) ? w.sum_dc[b] : 0ull;
  const uint32_t* pp = reinterpret_cast<const uint32_t*>(w.codes) + pair_index(b, g.P, 0);
  uint32_t* slot = w.etmp + (active ? b : 0) * slot_words_of(g);
  Extra<T> ex = {nullptr, 0, nullptr, kNoTrunc};
  if (CMP && active) {
    ex.kq = static_cast<const int*>(w.coefT) + 4 * b;
    ex.nco = reg ? g.ndim + 1 : 0;
    ex.up = static_cast<const T*>(w.ustage) + code_index(b, g.P, 0);
    ex.texp = bound_exponent<T>((T)st->eb);
  }
  EncRes e = {0u, 0u, 0u, 0ull, {0u, 0u, 0u, 0u}};
  if ((b & ~uint64_t(31)) < g.nb)  // a warp with blocks in the field (its pair rows exist)
    e = encode_codes<ABFT, false, CMP, T>(pp, P, slot, cb, cw0, g.R, 0u, 0u, ex, pairs_of(g.P), ring);
  if (active) {
    uint32_t kfix = 0xffffffffu, vfix = 0;
    bool bad = false;
    if (ABFT && (e.sq != sq_ref || e.isq != isq_ref)) {
      long long delta = 0;
      const long long m = locate_word(sq_ref, isq_ref, e.sq, e.isq, P, 0, &delta);
      bool fixed = false;
      if (m >= 0) {
        const uint32_t old = (pp[32 * (uint64_t)(m >> 1)] >> (16 * (m & 1))) & 0xffffu;
        const long long nv = (long long)old - delta;
        if (nv >= 0 && nv < (long long)g.bins) {
          kfix = (uint32_t)m;
          vfix = (uint32_t)nv;
          e = encode_codes<ABFT, true, CMP, T>(pp, P, slot, cb, cw0, g.R, kfix, vfix, ex, pairs_of(g.P));  // repaired
          fixed = true;
        }
      }
      if (fixed) {
        atomicAdd(&st->codes_corrected, 1ull);
      } else {
        bad = true;
        atomicAdd(&st->uncorrectable, 1ull);
        if (field) {  // every point the corrupted codes call unpredictable takes its input value
          const Box x = block_box(g, b);
          T* up = static_cast<T*>(w.ustage) + code_index(b, g.P, 0);
          for (uint32_t k = 0; k < P; ++k) {
            const uint32_t c = (pp[32 * (uint64_t)(k >> 1)] >> (16 * (k & 1))) & 0xffffu;
            if (c == 0) {
              const uint32_t l = k % x.e[2], q = k / x.e[2];
              up[32 * (uint64_t)k] = field[row_base(g, x, q / x.e[1], q % x.e[1]) + l];
            }
          }
          if (CMP)  // the compact payload carries the values: encoded again with them
            e = encode_codes<ABFT, false, CMP, T>(pp, P, slot, cb, cw0, g.R, 0u, 0u, ex, pairs_of(g.P));
        }
      }
    }
    // unpredictable values to the front of the block's staging slot, in order (in place: the
    // j-th value moves down from its point k >= j); the compact encoding has them in the payload
    if (!CMP) {
      T* up = static_cast<T*>(w.ustage) + code_index(b, g.P, 0);
      if (e.nun <= kPosKept) {
#pragma unroll
        for (uint32_t j = 0; j < kPosKept; ++j)
          if (j < e.nun && e.pos[j] != j) up[32 * (uint64_t)j] = up[32 * (uint64_t)e.pos[j]];
      } else {
        uint32_t j = 0;
        for (uint32_t k = 0; k < P; ++k) {
          uint32_t c = (pp[32 * (uint64_t)(k >> 1)] >> (16 * (k & 1))) & 0xffffu;
          if (k == kfix) c = vfix;
          if (c == 0) {
            if (j != k) up[32 * (uint64_t)j] = up[32 * (uint64_t)k];
            ++j;
          }
        }
      }
    }
    nbytes = (uint16_t)((e.bits + 7u) >> 3);
    const uint64_t fb = sh.boff + b;  // the block's index in the field
    *reinterpret_cast<uint16_t*>(out + L.sizes + 2 * fb) = (uint16_t)nbytes;
    *reinterpret_cast<uint16_t*>(out + L.ucounts + 2 * fb) = (uint16_t)e.nun;
    nun_enc = e.nun;
    if (ABFT) *reinterpret_cast<unsigned long long*>(out + L.sumdc + 8 * fb) = sdc_ref;
    // a block whose codes could not be repaired is reported in the header status word (by the
    // header's writer, from every shard's count, in a sharded field)
    if (bad && !sh.on) atomicOr(reinterpret_cast<unsigned int*>(out + 112), 1u);
  }
  // regression bitmap word of this warp's 32 blocks; the warp's unpredictable count; the
  // warp's share of its group's totals (the 32 blocks lie in one group of kGroup)
  const unsigned int ballot = __ballot_sync(0xffffffffu, active && reg);
  unsigned long long wun = warp_sum(nun_enc);
  const unsigned long long wtot = warp_sum(active ? pack_tot(nbytes, nun_enc, reg ? 1u : 0u) : 0ull);
  if (lane == 0 && b < g.nb) {
    if (!sh.on) {
      *reinterpret_cast<uint32_t*>(out + L.bitmap + 4 * (b >> 5)) = ballot;
    } else if (ballot) {  // a shard's 32 blocks may straddle two bitmap words of the field
      const uint64_t fb = sh.boff + (b & ~uint64_t(31));
      unsigned int* bw = reinterpret_cast<unsigned int*>(out + L.bitmap) + (fb >> 5);
      const uint32_t r = (uint32_t)(fb & 31);
      atomicOr(bw, ballot << r);
      if (r && (ballot >> (32 - r))) atomicOr(bw + 1, ballot >> (32 - r));
    }
    if (wun) atomicAdd(&st->n_unpred_enc, wun);
    const uint64_t gid = b / kGroup, ng = (g.nb + kGroup - 1) / kGroup;
    atomicAdd(&w.gt[gid], wtot);
    unsigned long long* sg = w.gt + ng + 2 * (gid / kSuper);
    atomicAdd(&sg[0], wtot & kMaskBytes);
    atomicAdd(&sg[1], (((wtot >> 25) & kMaskUn) << 17) | (wtot >> 46));
  }
}

template <typename T, bool ABFT, bool CMP>
__global__ void __launch_bounds__(128) k_encode_blocks(const T* __restrict__ field, Geo g, Ws w,
                                                       uint8_t* __restrict__ out) {
  __shared__ uint32_t cb_s[kCbWindow];
  __shared__ __align__(16) uint32_t ring_s[kRing * 8 * kRingStride];
  if (cta_failed(w.st)) return;
  cb_load(cb_s, g, w);
  __syncthreads();
  encode_block<T, ABFT, CMP>(g, w, out, cb_s, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, ring_s + threadIdx.x,
                             Shard{}, field);
}

// ---------------------------------------------------------------- K4b
template <typename T>
__device__ __forceinline__ void assemble_group(const Geo& g, const Ws& w, uint8_t* __restrict__ out, uint64_t cap,
                                               uint64_t gid, const Shard& sh = Shard{}) {
  __shared__ unsigned long long s_wt[8][3];
  __shared__ unsigned long long s_pre[8][3];
  __shared__ unsigned long long s_excl[3];
  __shared__ unsigned long long s_tot[3];
  State* st = w.st;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  const uint64_t b = gid * kGroup + tid;
  const bool active = b < g.nb;
  // The unpredictable section holds the points whose code, as encoded, is 0: the count K2 took
  // unless a block's codes could not be repaired. The payload follows that section (which the
  // compact encoding leaves empty).
  const unsigned long long n_unpred = sh.on ? sh.tot[1] : st->n_unpred_enc;
  const uint64_t s_dt = g.dtype ? 8 : 4;
  Layout L = st->L;
  L.payload = align16(L.unpred + (g.enc ? 0 : s_dt * n_unpred));
  // the group's exclusive prefix: the totals of the earlier super-groups and of the earlier
  // groups of its own super-group (summed by K4a, complete when this kernel starts), read
  // straight from memory without waiting on other CTAs; loaded first, so that these loads and
  // the slot's are in flight together
  // (each thread's first super-group and group entries are only loaded here and added after
  // the slot loads below have been issued; a field of up to 2^24 blocks has no more)
  unsigned long long pre[3] = {0, 0, 0};
  const uint64_t s0 = gid / kSuper;
  unsigned long long sga = 0, sgb = 0, gtv = 0;
  if (tid < s0) {
    sga = w.gt[ngroups + 2 * tid];
    sgb = w.gt[ngroups + 2 * tid + 1];
  }
  if (s0 * kSuper + tid < gid) gtv = w.gt[s0 * kSuper + tid];
  uint32_t bytes = 0, nun = 0;
  bool reg = false;
  // the first 64 bytes of the block's payload slot, loaded with its sizes: the slot does not
  // depend on the scan, only where it goes does
  const uint32_t n4 = (uint32_t)(slot_words_of(g) / 4);  // 16-byte pieces in a slot
  const uint4* src4 = reinterpret_cast<const uint4*>(w.etmp + b * slot_words_of(g));
  uint4 head[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) head[q] = (active && (uint32_t)q < n4) ? src4[q] : make_uint4(0u, 0u, 0u, 0u);
  if (active) {
    bytes = *reinterpret_cast<const uint16_t*>(out + L.sizes + 2 * (sh.boff + b));
    nun = *reinterpret_cast<const uint16_t*>(out + L.ucounts + 2 * (sh.boff + b));
    reg = w.flags[b] & 1;
  }
  pre[0] = sga + (gtv & kMaskBytes);
  pre[1] = (sgb >> 17) + ((gtv >> 25) & kMaskUn);
  pre[2] = (sgb & 0x1ffffull) + (gtv >> 46);
  for (uint64_t p = tid + blockDim.x; p < s0; p += blockDim.x) {  // larger fields: the rest
    const unsigned long long* sg = w.gt + ngroups + 2 * p;
    pre[0] += sg[0];
    pre[1] += sg[1] >> 17;
    pre[2] += sg[1] & 0x1ffffull;
  }
  for (uint64_t p = s0 * kSuper + tid + blockDim.x; p < gid; p += blockDim.x) {
    const unsigned long long t = w.gt[p];
    pre[0] += t & kMaskBytes;
    pre[1] += (t >> 25) & kMaskUn;
    pre[2] += t >> 46;
  }

  // CTA exclusive scan of (bytes, unpredictables, regression flag)
  unsigned long long v[3] = {bytes, nun, reg ? 1ull : 0ull}, inc[3] = {v[0], v[1], v[2]};
  for (int o = 1; o < 32; o <<= 1)
    for (int q = 0; q < 3; ++q) {
      unsigned long long nb = __shfl_up_sync(0xffffffffu, inc[q], o);
      if (lane >= (uint32_t)o) inc[q] += nb;
    }
  if (lane == 31)
    for (int q = 0; q < 3; ++q) s_wt[wid][q] = inc[q];
  for (int q = 0; q < 3; ++q) pre[q] = warp_sum(pre[q]);
  if (lane == 0)
    for (int q = 0; q < 3; ++q) s_pre[wid][q] = pre[q];
  __syncthreads();
  if (tid == 0) {
    unsigned long long run[3] = {0, 0, 0}, excl[3] = {0, 0, 0};
    for (int q2 = 0; q2 < 8; ++q2)
      for (int q = 0; q < 3; ++q) {
        const unsigned long long t = s_wt[q2][q];
        s_wt[q2][q] = run[q];
        run[q] += t;
        excl[q] += s_pre[q2][q];
      }
    for (int q = 0; q < 3; ++q) {
      s_tot[q] = run[q];
      s_excl[q] = excl[q];
    }
  }
  __syncthreads();

  if (tid == 0 && !sh.on) {
    const uint64_t go = L.groups + 24 * gid;
    for (int q = 0; q < 3; ++q) *reinterpret_cast<unsigned long long*>(out + go + 8 * q) = s_excl[q];
    if (gid == ngroups - 1) {
      const unsigned long long pay = s_excl[0] + s_tot[0];
      *reinterpret_cast<unsigned long long*>(out + 88) = n_unpred;
      *reinterpret_cast<unsigned long long*>(out + 96) = pay;
      *reinterpret_cast<unsigned long long*>(out + 104) = L.payload + pay;
      for (uint64_t o = L.unpred + (g.enc ? 0 : s_dt * n_unpred); o < L.payload && o < cap; ++o) out[o] = 0;  // gap
      st->n_unpred = n_unpred;
      st->L = L;
      st->payload_bytes = pay;
      st->total_bytes = L.payload + pay;
      if (L.payload + pay > cap) atomicOr(&st->error, ERR_CAPACITY);
    }
  }
  if (sh.on && sh.header && gid == 0 && tid == 0) {  // the field's totals, from every shard's
    const unsigned long long pay = sh.tot[0];
    *reinterpret_cast<unsigned long long*>(out + 88) = n_unpred;
    *reinterpret_cast<unsigned long long*>(out + 96) = pay;
    *reinterpret_cast<unsigned long long*>(out + 104) = L.payload + pay;
    *reinterpret_cast<unsigned int*>(out + 112) = sh.tot[3] ? 1u : 0u;
  }
  if (sh.on && tid == 0) {
    st->n_unpred = n_unpred;
    st->L = L;
    st->payload_bytes = sh.tot[0];
    st->total_bytes = L.payload + sh.tot[0];
    if (L.payload + sh.tot[0] > cap) atomicOr(&st->error, ERR_CAPACITY);
  }
  if (!active) return;

  // this block's offsets in the field's stream (the earlier shards' totals first)
  const unsigned long long pay_off = sh.pre[0] + s_excl[0] + s_wt[wid][0] + inc[0] - v[0];
  const unsigned long long un_off = sh.pre[1] + s_excl[1] + s_wt[wid][1] + inc[1] - v[1];
  const unsigned long long rg_off = sh.pre[2] + s_excl[2] + s_wt[wid][2] + inc[2] - v[2];
  if (sh.on && (sh.boff + b) % kGroup == 0) {  // the first block of a group of the field: its entry
    unsigned long long* ge = reinterpret_cast<unsigned long long*>(out + L.groups + 24 * ((sh.boff + b) / kGroup));
    ge[0] = pay_off;
    ge[1] = un_off;
    ge[2] = rg_off;
  }
  if (reg && !g.enc) {
    const T* cT = static_cast<const T*>(w.coefT) + 4 * b;
    T* dst = reinterpret_cast<T*>(out + L.coef) + (uint64_t)(g.ndim + 1) * rg_off;
    for (int a = 0; a <= g.ndim; ++a) dst[a] = cT[a];
  }
  // unpredictable values, moved by K4a to the front of the block's staging slot
  if (!g.enc) {
    const T* up = static_cast<const T*>(w.ustage) + code_index(b, g.P, 0);
    T* udst = reinterpret_cast<T*>(out + L.unpred);
    const unsigned long long ulim = n_unpred;
    for (uint32_t j = 0; j < nun; ++j)
      if (un_off + j < ulim) udst[un_off + j] = up[32 * (uint64_t)j];
  }
  // payload: stream bytes [lo, hi) = slot bytes [0, bytes). The stream word at wa = wa0 + 4i
  // holds slot bytes 4i - r .. 4i - r + 3 (r = lo mod 4): the top r bytes of slot word i - 1
  // and the low 4 - r bytes of slot word i. Words wholly inside [lo, hi) are stored whole;
  // the first and last are shared with the neighbouring blocks and written byte by byte.
  const uint64_t lo = L.payload + pay_off, hi = lo + bytes;
  if (hi > cap) {
    atomicOr(&st->error, ERR_CAPACITY);
    return;
  }
  // The slot is read 64 bytes (four aligned 16-byte loads, issued together) at a time, the first
  // 64 already in `head`, and the previous word carried.
  const uint32_t r = (uint32_t)(lo & 3), nw = (bytes + 3) / 4;
  const uint64_t wa0 = lo - r;
  const uint32_t nout = (uint32_t)((hi - wa0 + 3) >> 2);  // stream words touched
  uint32_t prev = 0;
  for (uint32_t i0 = 0; i0 < nout; i0 += 16) {
    uint4 q4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t pi = (i0 >> 2) + q;
      q4[q] = i0 == 0 ? head[q] : ((pi < n4 && 4 * pi < nw) ? src4[pi] : make_uint4(0u, 0u, 0u, 0u));
    }
    const uint32_t cur[16] = {q4[0].x, q4[0].y, q4[0].z, q4[0].w, q4[1].x, q4[1].y, q4[1].z, q4[1].w,
                              q4[2].x, q4[2].y, q4[2].z, q4[2].w, q4[3].x, q4[3].y, q4[3].z, q4[3].w};
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const uint32_t i = i0 + t;
      if (i >= nout) break;
      const uint32_t c = i < nw ? cur[t] : 0u;
      const uint32_t val = r ? __funnelshift_l(prev, c, 8 * r) : c;
      prev = c;
      const uint64_t wa = wa0 + 4 * (uint64_t)i;
      if (wa >= lo && wa + 4 <= hi) *reinterpret_cast<uint32_t*>(out + wa) = val;
      else put_bytes(out, wa, val, lo, hi);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 3) k_encode_assemble(Geo g, Ws w, uint8_t* __restrict__ out, uint64_t cap) {
  if (cta_failed(w.st)) return;
  assemble_group<T>(g, w, out, cap, blockIdx.x);
}

// A shard of a field (see Shard).
template <typename T, bool ABFT, bool CMP>
__global__ void __launch_bounds__(128) k_encode_blocks_shard(Geo g, Ws w, uint8_t* __restrict__ out, Shard sh) {
  __shared__ uint32_t cb_s[kCbWindow];
  __shared__ __align__(16) uint32_t ring_s[kRing * 8 * kRingStride];
  if (cta_failed(w.st)) return;
  cb_load(cb_s, g, w);
  __syncthreads();
  encode_block<T, ABFT, CMP>(g, w, out, cb_s, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, ring_s + threadIdx.x,
                             sh);
}

template <typename T>
__global__ void __launch_bounds__(256, 3) k_encode_assemble_shard(Geo g, Ws w, uint8_t* __restrict__ out, uint64_t cap,
                                                                   Shard sh) {
  if (cta_failed(w.st)) return;
  assemble_group<T>(g, w, out, cap, blockIdx.x, sh);
}

// ---------------------------------------------------------------- batches
template <typename T, bool ABFT>
__global__ void __launch_bounds__(128, ABFT ? 4 : 6) k_encode_blocks_batch(BatchArgs a) {
  __shared__ uint32_t cb_s[kCbWindow];
  __shared__ __align__(16) uint32_t ring_s[kRing * 8 * kRingStride];
  __shared__ Job s_job;
  batch_loop(
      a, s_job,
      [&] {
        cb_load(cb_s, s_job.g, s_job.w);
        __syncthreads();
      },
      [&](uint64_t it) {
        if (s_job.g.enc)
          encode_block<T, ABFT, true>(s_job.g, s_job.w, s_job.out, cb_s, it * blockDim.x + threadIdx.x,
                                      ring_s + threadIdx.x, Shard{}, static_cast<const T*>(s_job.field));
        else
          encode_block<T, ABFT, false>(s_job.g, s_job.w, s_job.out, cb_s, it * blockDim.x + threadIdx.x,
                                       ring_s + threadIdx.x, Shard{}, static_cast<const T*>(s_job.field));
      },
      NoOp());
}

template <typename T>
__global__ void __launch_bounds__(256) k_encode_assemble_batch(BatchArgs a) {
  __shared__ Job s_job;
  batch_loop(
      a, s_job, NoOp(), [&](uint64_t it) { assemble_group<T>(s_job.g, s_job.w, s_job.out, s_job.cap, it); }, NoOp());
}

template <class K>
unsigned batch_grid_of(K kern, uint32_t threads, uint64_t items, const Launch& L) {
  const int occ = occupancy(reinterpret_cast<const void*>(kern), (int)threads, 0);
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(items, (uint64_t)occ * L.sms));
}

template <typename T, bool ABFT>
void batch_blocks_t(const BatchArgs& a, const Launch& L) {
  auto kern = k_encode_blocks_batch<T, ABFT>;
  kern<<<batch_grid_of(kern, 128, a.start[a.n], L), 128, 0, L.stream>>>(a);
  note_launch();
}

template <typename T>
void batch_assemble_t(const BatchArgs& a, const Launch& L) {
  auto kern = k_encode_assemble_batch<T>;
  kern<<<batch_grid_of(kern, 256, a.start[a.n], L), 256, 0, L.stream>>>(a);
  note_launch();
}

template <typename T, bool ABFT>
void launch_encode_t(const void* field, const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L) {
  const uint64_t nchunks = (g.nb + 127) / 128, ngroups = (g.nb + kGroup - 1) / kGroup;
  if (!ngroups) return;
  const T* f = static_cast<const T*>(field);
  if (g.enc) k_encode_blocks<T, ABFT, true><<<(unsigned)nchunks, 128, 0, L.stream>>>(f, g, w, out);
  else k_encode_blocks<T, ABFT, false><<<(unsigned)nchunks, 128, 0, L.stream>>>(f, g, w, out);
  note_launch();
  k_encode_assemble<T><<<(unsigned)ngroups, 256, 0, L.stream>>>(g, w, out, cap);
  note_launch();
}

}  // namespace

uint64_t encode_slot_words(const Geo& g) { return slot_words_of(g); }

// items: 128-block chunks
void batch_encode_blocks(int dtype, bool abft, const BatchArgs& a, const Launch& L) {
  if (dtype == 0) {
    if (abft) batch_blocks_t<float, true>(a, L);
    else batch_blocks_t<float, false>(a, L);
  } else {
    if (abft) batch_blocks_t<double, true>(a, L);
    else batch_blocks_t<double, false>(a, L);
  }
}

// items: 256-block groups
void batch_encode_assemble(int dtype, const BatchArgs& a, const Launch& L) {
  if (dtype == 0) batch_assemble_t<float>(a, L);
  else batch_assemble_t<double>(a, L);
}

void launch_encode_shard_blocks(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Shard& sh,
                                const Launch& L) {
  (void)cap;
  const unsigned nchunks = (unsigned)((g.nb + 127) / 128);
  if (!nchunks) return;
  if (g.dtype == 0) {
    if (g.enc) {
      if (g.abft) k_encode_blocks_shard<float, true, true><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
      else k_encode_blocks_shard<float, false, true><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
    } else {
      if (g.abft) k_encode_blocks_shard<float, true, false><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
      else k_encode_blocks_shard<float, false, false><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
    }
  } else {
    if (g.enc) {
      if (g.abft) k_encode_blocks_shard<double, true, true><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
      else k_encode_blocks_shard<double, false, true><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
    } else {
      if (g.abft) k_encode_blocks_shard<double, true, false><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
      else k_encode_blocks_shard<double, false, false><<<nchunks, 128, 0, L.stream>>>(g, w, out, sh);
    }
  }
  note_launch();
}

void launch_encode_shard_assemble(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Shard& sh,
                                  const Launch& L) {
  const unsigned ngroups = (unsigned)((g.nb + kGroup - 1) / kGroup);
  if (!ngroups) return;
  if (g.dtype == 0) k_encode_assemble_shard<float><<<ngroups, 256, 0, L.stream>>>(g, w, out, cap, sh);
  else k_encode_assemble_shard<double><<<ngroups, 256, 0, L.stream>>>(g, w, out, cap, sh);
  note_launch();
}

void launch_encode(const void* field, const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L) {
  if (g.dtype == 0) {
    if (g.abft) launch_encode_t<float, true>(field, g, w, out, cap, L);
    else launch_encode_t<float, false>(field, g, w, out, cap, L);
  } else {
    if (g.abft) launch_encode_t<double, true>(field, g, w, out, cap, L);
    else launch_encode_t<double, false>(field, g, w, out, cap, L);
  }
}

}  // namespace sdcsz
