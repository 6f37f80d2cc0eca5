// K4: per-block Huffman encoding and stream assembly (the encoding and output steps of
// Algorithm 1 of the paper, without the Zstd stage).
//
// One CTA per random-access group of 256 blocks, one thread per block. Pass 1 reads the
// block's codes, checks them against sum_q/isum_q (Algorithm 1's check of the bin array before
// encoding: a single corrupted code is located and repaired) and sums the code lengths. A CTA scan plus a single-pass decoupled look-back
// across groups (group ids taken from a ticket in launch order, every wait bounded) gives each
// block its payload, unpredictable-value and coefficient offsets. Pass 2 re-reads the codes
// (L2 resident) and packs the bits MSB-first into 32-bit words: words wholly inside the
// block's byte range are stored whole, the partial first and last words byte by byte.
#include <algorithm>

#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

constexpr unsigned long long kFlagAgg = 1ull, kMaskBytes = (1ull << 22) - 1, kMaskUn = (1ull << 21) - 1;
constexpr uint32_t kCbWindow = 2048;  // codebook entries around the centre kept in shared memory

__device__ __forceinline__ unsigned long long pack_agg(unsigned long long bytes, unsigned long long un,
                                                       unsigned long long rg) {
  return (kFlagAgg << 62) | (rg << 43) | (un << 22) | bytes;
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

// Store the 32-bit big-endian word `v` at aligned word address `wa` of the stream, keeping
// only the bytes inside [lo, hi).
__device__ __forceinline__ void put_word(uint8_t* out, uint64_t wa, uint32_t v, uint64_t lo, uint64_t hi, bool fits) {
  if (!fits) return;
  if (wa >= lo && wa + 4 <= hi) {
    *reinterpret_cast<uint32_t*>(out + wa) = __byte_perm(v, 0, 0x0123);
  } else {
    for (int q = 0; q < 4; ++q)
      if (wa + q >= lo && wa + q < hi) out[wa + q] = (uint8_t)(v >> (24 - 8 * q));
  }
}

}  // namespace

__device__ __forceinline__ uint32_t cb_lo(const Geo& g) { return g.R > kCbWindow / 2 ? g.R - kCbWindow / 2 : 0; }

// Shared-memory window of the codebook around the centre bin.
__device__ __forceinline__ void cb_load(uint32_t* cb_s, const Geo& g, const Ws& w) {
  const uint32_t lo = cb_lo(g);
  for (uint32_t q = threadIdx.x; q < kCbWindow; q += blockDim.x)
    cb_s[q] = lo + q < g.bins ? __ldg(&w.codebook[lo + q]) : 0u;
}

// One random-access group (256 blocks, one per thread) of the stream.
template <typename T, bool ABFT>
__device__ __forceinline__ void encode_group(const Geo& g, const Ws& w, uint8_t* __restrict__ out, uint64_t cap,
                                             uint64_t gid, const uint32_t* cb_s) {
  __shared__ unsigned long long s_wt[8][3];
  __shared__ unsigned long long s_excl[3];
  __shared__ unsigned long long s_tot[3];
  State* st = w.st;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  Codebook cb;
  cb.lo = cb_lo(g);
  cb.s = cb_s;
  cb.g = w.codebook;
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  const uint64_t b = gid * kGroup + tid;
  const bool active = b < g.nb;
  const Layout L = st->L;
  const uint32_t* __restrict__ codes = reinterpret_cast<const uint32_t*>(w.codes);

  // pass 1: verify codes, count bits and unpredictables
  uint32_t P = 0, bits = 0, nun = 0, kfix = 0xffffffffu, vfix = 0;
  bool reg = false, bad = false;
  if (active) {
    P = block_box(g, b).P;
    reg = w.flags[b] & 1;
    uint32_t s = 0;
    unsigned long long is = 0;
    const uint32_t* pp = codes + pair_index(b, g.P, 0);
    const uint32_t P2 = P >> 1;
    // isum over a pair: (2m+1) c0 + (2m+2) c1 = (2m+1)(c0 + c1) + c1
    auto pair = [&](uint32_t wp2, uint32_t k2) {
      const uint32_t c0 = wp2 & 0xffffu, c1 = wp2 >> 16;
      bits += (cb(c0) & 31u) + (cb(c1) & 31u);
      nun += (c0 == 0) + (c1 == 0);
      if (ABFT) {
        s += c0 + c1;
        mad_wide(is, c0 + c1, 2 * k2 + 1);
        is += c1;
      }
    };
    // eight independent loads in flight per thread, then their arithmetic
    uint32_t k2 = 0;
    for (; k2 + 8 <= P2; k2 += 8) {
      uint32_t wq[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) wq[q] = pp[32 * (uint64_t)(k2 + q)];
#pragma unroll
      for (int q = 0; q < 8; ++q) pair(wq[q], k2 + q);
    }
    for (; k2 < P2; ++k2) pair(pp[32 * (uint64_t)k2], k2);
    if (P & 1) {  // odd point count: the last pair holds one code
      const uint32_t c0 = pp[32 * (uint64_t)P2] & 0xffffu;
      bits += cb(c0) & 31u;
      nun += (c0 == 0);
      if (ABFT) {
        s += c0;
        mad_wide(is, c0, P);
      }
    }
    if (ABFT && (s != w.sum_q[b] || is != w.isum_q[b])) {
      long long delta = 0;
      const long long m = locate_word(w.sum_q[b], w.isum_q[b], s, is, P, 0, &delta);
      bool fixed = false;
      if (m >= 0) {
        const uint32_t old = (pp[32 * (uint64_t)(m >> 1)] >> (16 * (m & 1))) & 0xffffu;
        const long long nv = (long long)old - delta;
        if (nv >= 0 && nv < (long long)g.bins) {
          kfix = (uint32_t)m;
          vfix = (uint32_t)nv;
          bits += (cb(vfix) & 31u) - (cb(old) & 31u);
          nun += (vfix == 0) - (old == 0);
          fixed = true;
        }
      }
      if (fixed) atomicAdd(&st->codes_corrected, 1ull);
      else {
        bad = true;
        atomicAdd(&st->uncorrectable, 1ull);
      }
    }
  }
  const unsigned long long bytes = (bits + 7u) >> 3;

  // CTA exclusive scan of (bytes, unpredictables, regression flag)
  unsigned long long v[3] = {bytes, nun, reg ? 1ull : 0ull}, inc[3] = {v[0], v[1], v[2]};
  for (int o = 1; o < 32; o <<= 1)
    for (int q = 0; q < 3; ++q) {
      unsigned long long nb = __shfl_up_sync(0xffffffffu, inc[q], o);
      if (lane >= (uint32_t)o) inc[q] += nb;
    }
  if (lane == 31)
    for (int q = 0; q < 3; ++q) s_wt[wid][q] = inc[q];
  __syncthreads();
  if (wid == 0) {
    // warp totals -> exclusive prefixes (lane 0), then a warp-wide decoupled look-back
    unsigned long long run[3] = {0, 0, 0};
    if (lane == 0) {
      for (int q2 = 0; q2 < 8; ++q2)
        for (int q = 0; q < 3; ++q) {
          const unsigned long long t = s_wt[q2][q];
          s_wt[q2][q] = run[q];
          run[q] += t;
        }
      for (int q = 0; q < 3; ++q) s_tot[q] = run[q];
    }
    for (int q = 0; q < 3; ++q) run[q] = __shfl_sync(0xffffffffu, run[q], 0);
    LookBack* me = &w.lb[gid];
    unsigned long long excl[3] = {0, 0, 0};
    if (gid > 0 && lane == 0) {
      *(volatile unsigned long long*)&me->agg = pack_agg(run[0], run[1], run[2]);
      __threadfence();
    }
    // lane l looks at predecessor gid-1-l-32r; the nearest one with an inclusive prefix ends it
    bool finished = gid == 0;
    for (int64_t base = (int64_t)gid - 1; !finished; base -= 32) {
      const int64_t p = base - (int64_t)lane;
      unsigned long long va[3] = {0, 0, 0};
      bool incl = p < 0, ready = p < 0;
      uint32_t spins = 0;
      while (true) {
        if (!ready) {
          const LookBack* pr = &w.lb[p];
          if (*(volatile const unsigned int*)&pr->incl_flag) {
            __threadfence();
            va[0] = *(volatile const unsigned long long*)&pr->incl[0];
            va[1] = *(volatile const unsigned long long*)&pr->incl[1];
            va[2] = *(volatile const unsigned long long*)&pr->incl[2];
            incl = ready = true;
          } else {
            const unsigned long long a = *(volatile const unsigned long long*)&pr->agg;
            if (a >> 62) {
              va[0] = a & kMaskBytes;
              va[1] = (a >> 22) & kMaskUn;
              va[2] = (a >> 43) & 0x7ffffull;
              ready = true;
            }
          }
        }
        if (__all_sync(0xffffffffu, ready)) break;
        if (++spins > kSpinLimit) {
          if (lane == 0) atomicOr(&st->error, ERR_TIMEOUT);
          ready = incl = true;  // give up: the stream is then reported as failed
        }
        __nanosleep(32);
      }
      // lanes up to the nearest inclusive prefix contribute
      const unsigned int im = __ballot_sync(0xffffffffu, incl);
      const uint32_t stop = im ? (uint32_t)(__ffs(im) - 1) : 31u;
      for (int q = 0; q < 3; ++q) {
        unsigned long long c = lane <= stop ? va[q] : 0ull;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl[q] += c;
      }
      finished = im != 0;
    }
    if (lane == 0) {
      me->incl[0] = excl[0] + run[0];
      me->incl[1] = excl[1] + run[1];
      me->incl[2] = excl[2] + run[2];
      __threadfence();
      *(volatile unsigned int*)&me->incl_flag = 1u;
      for (int q = 0; q < 3; ++q) s_excl[q] = excl[q];
    }
  }
  __syncthreads();

  if (tid == 0) {
    const uint64_t go = L.groups + 24 * gid;
    for (int q = 0; q < 3; ++q) *reinterpret_cast<unsigned long long*>(out + go + 8 * q) = s_excl[q];
    if (gid == ngroups - 1) {
      const unsigned long long pay = s_excl[0] + s_tot[0];
      *reinterpret_cast<unsigned long long*>(out + 96) = pay;
      *reinterpret_cast<unsigned long long*>(out + 104) = L.payload + pay;
      st->payload_bytes = pay;
      st->total_bytes = L.payload + pay;
      if (L.payload + pay > cap) atomicOr(&st->error, ERR_CAPACITY);
    }
  }
  // bitmap word of this warp's 32 blocks
  const unsigned int ballot = __ballot_sync(0xffffffffu, active && reg);
  if (lane == 0 && (gid * kGroup + wid * 32) < g.nb)
    *reinterpret_cast<uint32_t*>(out + L.bitmap + 4 * ((gid * kGroup) / 32 + wid)) = ballot;
  if (!active) return;

  const unsigned long long pay_off = s_excl[0] + s_wt[wid][0] + inc[0] - v[0];
  const unsigned long long un_off = s_excl[1] + s_wt[wid][1] + inc[1] - v[1];
  const unsigned long long rg_off = s_excl[2] + s_wt[wid][2] + inc[2] - v[2];
  *reinterpret_cast<uint16_t*>(out + L.sizes + 2 * b) = (uint16_t)bytes;
  *reinterpret_cast<uint16_t*>(out + L.ucounts + 2 * b) = (uint16_t)nun;
  if (ABFT) *reinterpret_cast<unsigned long long*>(out + L.sumdc + 8 * b) = w.sum_dc[b];
  if (reg) {
    const T* cT = static_cast<const T*>(w.coefT) + 4 * b;
    T* dst = reinterpret_cast<T*>(out + L.coef) + (uint64_t)(g.ndim + 1) * rg_off;
    for (int a = 0; a <= g.ndim; ++a) dst[a] = cT[a];
  }
  // pass 2: pack the codes MSB-first; copy the unpredictable values in order. Every word
  // emitted inside the loop is whole and inside the block except the first one when the block
  // starts mid-word (its leading bytes belong to the previous block); the last, partial word
  // is written after the loop.
  const uint64_t lo = L.payload + pay_off, hi = lo + bytes;
  const bool fits = hi <= cap;
  if (!fits) atomicOr(&st->error, ERR_CAPACITY);
  uint64_t wa = lo & ~uint64_t(3);                  // aligned word being filled
  unsigned long long acc = 0;
  uint32_t nacc = 8u * (uint32_t)(lo & 3);          // leading bytes of the first word are not ours
  bool head = (lo & 3) != 0;
  const T* ust = static_cast<const T*>(w.ustage);
  T* udst = reinterpret_cast<T*>(out + L.unpred);
  unsigned long long uidx = un_off;
  const unsigned long long ulim = st->n_unpred;
  const uint32_t* pp = codes + pair_index(b, g.P, 0);
  const T* up = ust + code_index(b, g.P, 0);
  const uint32_t cw0 = __ldg(&w.codebook[0]);
  auto put = [&](uint32_t c, uint32_t k) {
    if (ABFT && k == kfix) c = vfix;
    const uint32_t cw = c ? cb(c) : cw0;
    const uint32_t len = cw & 31u;
    acc = (acc << len) | (cw >> 5);
    nacc += len;
    if (nacc >= 32) {
      nacc -= 32;
      const uint32_t word = (uint32_t)(acc >> nacc);
      if (head) {
        put_word(out, wa, word, lo, hi, fits);
        head = false;
      } else if (fits) {
        *reinterpret_cast<uint32_t*>(out + wa) = __byte_perm(word, 0, 0x0123);
      }
      wa += 4;
    }
    if (c == 0) {
      if (uidx < ulim) udst[uidx] = up[32 * (uint64_t)k];
      ++uidx;
    }
  };
  // code pairs loaded four at a time ahead of their use
  const uint32_t P2 = P >> 1;
  for (uint32_t k2 = 0; k2 < P2; k2 += 4) {
    uint32_t wq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) wq[q] = (k2 + q < P2) ? pp[32 * (uint64_t)(k2 + q)] : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (k2 + q < P2) {
        put(wq[q] & 0xffffu, 2 * (k2 + q));
        put(wq[q] >> 16, 2 * (k2 + q) + 1);
      }
    }
  }
  if (P & 1) put(pp[32 * (uint64_t)P2] & 0xffffu, P - 1);
  if (nacc) put_word(out, wa, (uint32_t)(acc << (32 - nacc)), lo, hi, fits);
  if (bad) {
    // a block whose codes could not be repaired is reported in the header status word
    atomicOr(reinterpret_cast<unsigned int*>(out + 112), 1u);
  }
}

template <typename T, bool ABFT>
__global__ void __launch_bounds__(256) k_encode(Geo g, Ws w, uint8_t* __restrict__ out, uint64_t cap) {
  __shared__ uint32_t s_gid;
  __shared__ uint32_t cb_s[kCbWindow];
  State* st = w.st;
  if (*(volatile unsigned int*)&st->error) return;
  if (threadIdx.x == 0) s_gid = atomicAdd(&st->ticket, 1u);
  cb_load(cb_s, g, w);
  __syncthreads();
  encode_group<T, ABFT>(g, w, out, cap, s_gid, cb_s);
}

// Batched: the groups of every job; a job's groups are pulled in increasing order, so each
// look-back only waits for groups already taken by running CTAs.
template <typename T, bool ABFT>
__global__ void __launch_bounds__(256) k_encode_batch(BatchArgs a) {
  __shared__ uint32_t cb_s[kCbWindow];
  __shared__ Job s_job;
  batch_loop(
      a, s_job,
      [&] {
        cb_load(cb_s, s_job.g, s_job.w);
        __syncthreads();
      },
      [&](uint64_t it) { encode_group<T, ABFT>(s_job.g, s_job.w, s_job.out, s_job.cap, it, cb_s); }, NoOp());
}

template <typename T, bool ABFT>
static void batch_encode_t(const BatchArgs& a, const Launch& L) {
  auto kern = k_encode_batch<T, ABFT>;
  const int occ = occupancy(reinterpret_cast<const void*>(kern), 256, 0);
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(a.start[a.n], (uint64_t)occ * L.sms));
  kern<<<grid, 256, 0, L.stream>>>(a);
  note_launch();
}

void batch_encode(int dtype, bool abft, const BatchArgs& a, const Launch& L) {
  if (dtype == 0) {
    if (abft) batch_encode_t<float, true>(a, L);
    else batch_encode_t<float, false>(a, L);
  } else {
    if (abft) batch_encode_t<double, true>(a, L);
    else batch_encode_t<double, false>(a, L);
  }
}

void launch_encode(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L) {
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  if (!ngroups) return;
  if (g.dtype == 0) {
    if (g.abft) k_encode<float, true><<<(unsigned)ngroups, 256, 0, L.stream>>>(g, w, out, cap);
    else k_encode<float, false><<<(unsigned)ngroups, 256, 0, L.stream>>>(g, w, out, cap);
  } else {
    if (g.abft) k_encode<double, true><<<(unsigned)ngroups, 256, 0, L.stream>>>(g, w, out, cap);
    else k_encode<double, false><<<(unsigned)ngroups, 256, 0, L.stream>>>(g, w, out, cap);
  }  note_launch();
}

}  // namespace sdcsz
