// K6 / K7: the lossless stage that ends Algorithm 1 and starts Algorithm 2 (Zstd in the paper).
//
// An order-0 range asymmetric numeral system (rANS) coder over the bytes from the sum_dc
// section to the end of the stream (sum_dc, coefficients, unpredictable values, payload); the
// header, code table and random-access tables stay as they are. Frequencies are the byte
// counts scaled to 4096; the bytes are cut into 16 KiB chunks, each coded by one warp with 32
// interleaved 32-bit states (byte i of a chunk belongs to lane i mod 32), 16-bit
// renormalisation. The warp runs over its chunk from the last group of 32 bytes to the first;
// the lanes that renormalise at a step emit one word each, placed (by a ballot) so that the
// decoder, which runs forward and takes words in increasing lane order at each step, reads them
// in sequence. Section: 256 u16 frequencies, u32 end offset of each chunk, then the chunks
// (32 final states, the words), each padded to 4 bytes.
//
// Compression: K6a byte histogram (warp-aggregated), K6b frequencies (one warp), K6c one warp
// per chunk into a per-chunk scratch slot, K6d one CTA scans the chunk sizes and writes the
// header and chunk table, K6e one warp per chunk places the coded chunks and the remaining CTAs
// copy the tables. Decompression: K7, one warp per chunk (and CTAs for the tables), into a
// scratch copy of the stream without the stage, which the decoder then reads.
#include <algorithm>

#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

constexpr uint32_t kRansLow = 1u << 16;

// ---------------------------------------------------------------- K6a
__global__ void __launch_bounds__(256) k_ll_hist(const uint8_t* __restrict__ raw, State* st,
                                                 unsigned long long* hist) {
  __shared__ unsigned int sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  const bool ok = *(volatile unsigned int*)&st->error == 0;
  const uint64_t from = st->L.sumdc, end = st->total_bytes;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 16;
  if (ok) {
    for (uint64_t q = from + ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16; q < end; q += stride) {
      uint32_t wv[4];
      if (q + 16 <= end) {  // from is 16-byte aligned, so is q
        const uint4 v = *reinterpret_cast<const uint4*>(raw + q);
        wv[0] = v.x;
        wv[1] = v.y;
        wv[2] = v.z;
        wv[3] = v.w;
      } else {
        for (int t = 0; t < 4; ++t) {
          wv[t] = 0;
          for (int u = 0; u < 4; ++u) {
            const uint64_t a = q + 4 * t + u;
            wv[t] |= (a < end ? (uint32_t)raw[a] : 0u) << (8 * u);
          }
        }
      }
      const uint32_t n = (uint32_t)min((uint64_t)16, end - q);
      const unsigned act = __activemask();
#pragma unroll
      for (uint32_t b = 0; b < 16; ++b) {
        // bytes past the end count as 256 (ignored); equal bytes of the warp add once
        const uint32_t v = b < n ? (wv[b >> 2] >> (8 * (b & 3))) & 0xffu : 256u;
        const unsigned same = __match_any_sync(act, v);
        if (v < 256 && (threadIdx.x & 31) == (uint32_t)(__ffs(same) - 1)) atomicAdd(&sh[v], (unsigned)__popc(same));
      }
    }
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)sh[threadIdx.x]);
}

// ---------------------------------------------------------------- K6b
// Frequencies (one warp; lane l owns bytes 8l .. 8l+7): scaled counts, at least 1 for a byte
// that occurs; the sum is brought to 4096 by taking one at a time from the largest frequency
// above 1 (ties: smaller byte), or giving the shortfall to the most frequent byte (ties:
// smaller byte). Writes the frequency table at the section start and the cumulative table.
__global__ void k_ll_freq(State* st, const unsigned long long* __restrict__ hist, uint8_t* out,
                          uint32_t* cum) {
  const uint32_t lane = threadIdx.x;
  if (*(volatile unsigned int*)&st->error) return;
  const uint64_t from = st->L.sumdc, end = st->total_bytes;
  if (lane == 0) st->raw_total = end;
  const uint64_t total = end > from ? end - from : 0;
  unsigned long long cnt[8];
  uint32_t f[8];
  long long sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    cnt[q] = hist[8 * lane + q];
    f[q] = 0;
    if (cnt[q] && total) {
      const unsigned long long v = cnt[q] * kLLM / total;
      f[q] = v < 1 ? 1u : (uint32_t)v;
    }
    sum += f[q];
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (total) {
    if (sum > (long long)kLLM) {
      // Taking one at a time from the largest frequency (smaller byte on ties) D = sum - 4096
      // times ends with every frequency above v capped at v, where v is the smallest level
      // whose cap removes at most D (A(v) = sum of max(0, f - v) <= D), and the R = D - A(v)
      // smallest bytes at level v taken down to v - 1 (v >= 2: A(1) >= 4096 - 256 > D).
      const long long D = sum - (long long)kLLM;
      auto above = [&](uint32_t v) {
        long long a = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) a += f[q] > v ? (long long)(f[q] - v) : 0;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        return a;
      };
      uint32_t lo = 1, hi = kLLM;  // A(hi) = 0 <= D; find the smallest v with A(v) <= D
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (above(mid) <= D) hi = mid;
        else lo = mid + 1;
      }
      const uint32_t v = lo;
      const long long R = D - above(v);
      uint32_t mine = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) mine += f[q] >= v;
      uint32_t incl = mine;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
      }
      uint32_t rank = incl - mine;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (f[q] >= v) {
          f[q] = (long long)rank < R ? v - 1 : v;
          ++rank;
        }
      sum = kLLM;
    }
    if (sum < (long long)kLLM) {
      // the most frequent byte, smaller byte on ties
      unsigned long long bc = 0;
      uint32_t bb = 256;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (bb == 256 || cnt[q] > bc) {
          bc = cnt[q];
          bb = 8 * lane + q;
        }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long oc = __shfl_xor_sync(0xffffffffu, bc, o);
        const uint32_t ob = __shfl_xor_sync(0xffffffffu, bb, o);
        if (oc > bc || (oc == bc && ob < bb)) {
          bc = oc;
          bb = ob;
        }
      }
      if (bb / 8 == lane) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if ((uint32_t)q == bb % 8) f[q] += (uint32_t)(kLLM - sum);
      }
    }
  }
  // table and cumulative sums (lane-exclusive prefix of the lane totals)
  uint32_t own = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) own += f[q];
  uint32_t incl = own;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += v;
  }
  uint32_t c = incl - own;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t b = 8 * lane + q;
    out[from + 2 * b] = (uint8_t)f[q];
    out[from + 2 * b + 1] = (uint8_t)(f[q] >> 8);
    cum[b] = c;
    c += f[q];
  }
  if (lane == 31) cum[256] = c;
}

// ---------------------------------------------------------------- K6c
// Per byte: cumulative frequency and frequency packed (c | f << 16), and m = ceil(2^32 / f)
// (0 for f = 1), so that x / f is umulhi(x, m) or one less (checked with the remainder).
__device__ __forceinline__ void ll_divmod(uint32_t x, uint32_t f, uint32_t m, uint32_t& q, uint32_t& r) {
  if (f == 1) {
    q = x;
    r = 0;
    return;
  }
  q = __umulhi(x, m);
  long long rr = (long long)x - (long long)q * f;
  if (rr < 0) {
    --q;
    rr += f;
  }
  r = (uint32_t)rr;
}

// One warp per chunk, from its last group of 32 bytes to its first. The bytes are read 128 at a
// time (lane l holds bytes 4l..4l+3 of a group of four steps), two groups ahead of their use,
// and handed to the lane that codes them with a shuffle.
__global__ void __launch_bounds__(256) k_ll_encode(const uint8_t* __restrict__ raw, State* st, Ws w) {
  __shared__ uint2 tab[256];
  for (uint32_t t = threadIdx.x; t < 256; t += blockDim.x) {
    const uint32_t c = w.llcum[t], f = w.llcum[t + 1] - c;
    tab[t] = make_uint2(c | (f << 16), f > 1 ? (uint32_t)((0x100000000ull + f - 1) / f) : 0u);
  }
  __syncthreads();
  if (*(volatile unsigned int*)&st->error) return;
  const uint64_t from = st->L.sumdc, end = st->raw_total;
  const uint64_t nch = ll_chunks(from, end);
  const uint64_t k = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (k >= nch) return;
  const uint64_t base = from + k * kLLChunk;  // 16-byte aligned
  const uint32_t n = (uint32_t)min((uint64_t)kLLChunk, end - base);
  uint16_t* slot = w.llw + k * kLLChunk;
  uint32_t x = kRansLow, top = kLLChunk;
  const uint32_t above = lane == 31 ? 0u : (0xffffffffu << (lane + 1));  // lanes above this one
  auto group = [&](int g) -> uint32_t {  // bytes 128 g + 4 lane .. + 3 of the chunk
    if (g < 0) return 0u;
    const uint32_t o = 128u * (uint32_t)g + 4u * lane;
    if (o + 4 <= n) return *reinterpret_cast<const uint32_t*>(raw + base + o);
    uint32_t v = 0;
    for (uint32_t u = 0; u < 4; ++u)
      if (o + u < n) v |= (uint32_t)raw[base + o + u] << (8 * u);
    return v;
  };
  const uint32_t T = (n + 31) / 32;
  const int G = (int)((T + 3) / 4);
  uint32_t cur = group(G - 1), nx1 = group(G - 2), nx2 = group(G - 3);
  for (int g = G - 1; g >= 0; --g) {
#pragma unroll
    for (int tt = 3; tt >= 0; --tt) {
      const uint32_t t = 4u * (uint32_t)g + (uint32_t)tt;
      if (t >= T) continue;  // warp-uniform
      const uint32_t i = t * 32 + lane;
      const bool act = i < n;
      const uint32_t wv = __shfl_sync(0xffffffffu, cur, 8 * tt + (lane >> 2));
      const uint32_t sbyte = (wv >> (8 * (lane & 3))) & 0xffu;
      const uint2 e = tab[sbyte];
      const uint32_t c = e.x & 0xffffu, f = e.x >> 16;
      const bool need = act && (unsigned long long)x >= ((unsigned long long)f << 20);
      const unsigned mask = __ballot_sync(0xffffffffu, need);
      if (need) {
        slot[top - 1 - __popc(mask & above)] = (uint16_t)(x & 0xffffu);
        x >>= 16;
      }
      top -= __popc(mask);
      if (act) {
        uint32_t q, r;
        ll_divmod(x, f, e.y, q, r);
        x = (q << kLLScale) + r + c;
      }
    }
    cur = nx1;
    nx1 = nx2;
    nx2 = group(g - 3);
  }
  w.llst[k * 32 + lane] = x;
  if (lane == 0) {
    w.llsz[k] = (128u + 2u * (kLLChunk - top) + 3u) & ~3u;
    w.lltop[k] = top;
  }
}

// ---------------------------------------------------------------- K6d
// One CTA: chunk offsets (exclusive scan of the sizes), the chunk end table, the coded total,
// the header of the coded stream.
__global__ void __launch_bounds__(1024) k_ll_scan(State* st, Ws w, uint8_t* out, uint64_t cap) {
  __shared__ unsigned long long part[1024];
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = *(volatile unsigned int*)&st->error != 0;
  __syncthreads();
  if (s_fail) return;
  const uint64_t from = st->L.sumdc, end = st->raw_total;
  const uint64_t nch = ll_chunks(from, end);
  const uint64_t data = ll_data(from, nch);
  const uint64_t per = (nch + blockDim.x - 1) / blockDim.x;
  const uint64_t b0 = threadIdx.x * per, b1 = min(nch, b0 + per);
  unsigned long long s = 0;
  for (uint64_t k = b0; k < b1; ++k) s += w.llsz[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (uint32_t o = 1; o < blockDim.x; o <<= 1) {
    const unsigned long long v = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  const unsigned long long total_chunks = part[blockDim.x - 1];
  const uint64_t coded = data + total_chunks;
  const bool fits = coded <= cap;
  unsigned long long run = part[threadIdx.x] - s;
  for (uint64_t k = b0; k < b1 && fits; ++k) {
    w.lloff[k] = data + run;
    run += w.llsz[k];
    const uint32_t e = (uint32_t)run;
    uint8_t* p = out + from + kLLTable + 4 * k;
    p[0] = (uint8_t)e;
    p[1] = (uint8_t)(e >> 8);
    p[2] = (uint8_t)(e >> 16);
    p[3] = (uint8_t)(e >> 24);
  }
  if (!fits) {
    if (threadIdx.x == 0) atomicOr(&st->error, ERR_CAPACITY);
    return;
  }
  // the gap before the chunks
  for (uint64_t o = from + kLLTable + 4 * nch + threadIdx.x; o < data; o += blockDim.x) out[o] = 0;
  // header: the stream's, with the stage flag, the coded total and the total without the stage
  if (threadIdx.x < kHeaderBytes) {
    const uint32_t q = threadIdx.x;
    uint8_t v = w.raw[q];
    if (q == 51) v |= 2;
    if (q >= 104 && q < 112) v = (uint8_t)(coded >> (8 * (q - 104)));
    if (q >= 120) v = (uint8_t)(end >> (8 * (q - 120)));
    out[q] = v;
  }
  if (threadIdx.x == 0) st->total_bytes = coded;
}

// ---------------------------------------------------------------- K6e
// Warps of the first CTAs: one chunk each (states, then the words in decoding order, then the
// padding); the CTAs after them copy the tables between the header and the section.
__global__ void __launch_bounds__(256) k_ll_place(State* st, Ws w, uint8_t* out, unsigned chunk_ctas) {
  if (*(volatile unsigned int*)&st->error) return;
  const uint64_t from = st->L.sumdc, end = st->raw_total;
  const uint64_t nch = ll_chunks(from, end);
  const uint32_t lane = threadIdx.x & 31;
  if (blockIdx.x < chunk_ctas) {
    const uint64_t k = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= nch) return;
    uint8_t* dst = out + w.lloff[k];
    reinterpret_cast<uint32_t*>(dst)[lane] = w.llst[k * 32 + lane];
    const uint32_t top = w.lltop[k], nw = kLLChunk - top;
    const uint16_t* src = w.llw + k * kLLChunk + top;
    uint16_t* dw = reinterpret_cast<uint16_t*>(dst + 128);
    for (uint32_t q = lane; q < nw; q += 32) dw[q] = src[q];
    if (lane == 0 && (nw & 1)) dw[nw] = 0;
    return;
  }
  const uint64_t t0 = ((uint64_t)(blockIdx.x - chunk_ctas) * blockDim.x + threadIdx.x) * 16 + kHeaderBytes;
  const uint64_t stride = (uint64_t)(gridDim.x - chunk_ctas) * blockDim.x * 16;
  for (uint64_t o = t0; o < from; o += stride)  // from and the header are 16-byte aligned
    *reinterpret_cast<uint4*>(out + o) = *reinterpret_cast<const uint4*>(w.raw + o);
}

// ---------------------------------------------------------------- K7
// Decompression: warps of the first CTAs decode one chunk each into `raw`; the CTAs after them
// copy the tables and write the header of the stream without the stage. A chunk whose end
// offsets or frequency table are impossible makes the stream malformed.
__global__ void __launch_bounds__(256) k_ll_unpack(const uint8_t* __restrict__ s, uint64_t nbytes, uint64_t from,
                                                   uint64_t raw_total, uint8_t* raw, State* st, unsigned chunk_ctas) {
  __shared__ uint32_t cum[257];
  __shared__ uint8_t sym[kLLM];
  const uint64_t nch = ll_chunks(from, raw_total);
  const uint64_t data = ll_data(from, nch);
  if (blockIdx.x >= chunk_ctas) {
    const uint64_t t0 = ((uint64_t)(blockIdx.x - chunk_ctas) * blockDim.x + threadIdx.x) * 16 + kHeaderBytes;
    const uint64_t stride = (uint64_t)(gridDim.x - chunk_ctas) * blockDim.x * 16;
    for (uint64_t o = t0; o < from; o += stride)
      *reinterpret_cast<uint4*>(raw + o) = *reinterpret_cast<const uint4*>(s + o);
    if (blockIdx.x == chunk_ctas && threadIdx.x < kHeaderBytes) {
      const uint32_t q = threadIdx.x;
      uint8_t v = s[q];
      if (q == 51) v &= 1;
      if (q >= 104 && q < 112) v = (uint8_t)(raw_total >> (8 * (q - 104)));
      if (q >= 120) v = 0;
      raw[q] = v;
    }
    return;
  }
  // frequency table: cumulative sums (one warp), then the slot -> byte table
  if (threadIdx.x < 32) {
    const uint32_t lane = threadIdx.x;
    uint32_t f[8], own = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint64_t a = from + 2 * (8 * lane + q);
      f[q] = (uint32_t)s[a] | ((uint32_t)s[a + 1] << 8);
      own += f[q];
    }
    uint32_t incl = own;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += v;
    }
    uint32_t c = incl - own;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      cum[8 * lane + q] = c;
      c += f[q];
    }
    if (lane == 31) cum[256] = c;
  }
  __syncthreads();
  const bool table_ok = nch == 0 || cum[256] == kLLM;
  for (uint32_t q = threadIdx.x; q < kLLM; q += blockDim.x) {
    uint32_t lo = 0, hi = 256;  // the byte b with cum[b] <= q < cum[b + 1]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (cum[mid] <= q) lo = mid;
      else hi = mid;
    }
    sym[q] = (uint8_t)lo;
  }
  __syncthreads();
  const uint64_t k = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (k >= nch) return;
  if (!table_ok) {
    if (lane == 0) atomicOr(&st->error, ERR_FORMAT);
    return;
  }
  const uint8_t* ends = s + from + kLLTable;
  auto end_of = [&](uint64_t q) {
    const uint8_t* p = ends + 4 * q;
    return (uint64_t)p[0] | ((uint64_t)p[1] << 8) | ((uint64_t)p[2] << 16) | ((uint64_t)p[3] << 24);
  };
  const uint64_t c0 = k ? end_of(k - 1) : 0, c1 = end_of(k);
  if (c1 < c0 || data + c1 > nbytes || ((data + c0) & 3)) {
    if (lane == 0) atomicOr(&st->error, ERR_FORMAT);
    return;
  }
  const uint8_t* chunk = s + data + c0;
  const uint64_t len = c1 - c0;
  uint32_t x = 4 * (lane + 1) <= len ? reinterpret_cast<const uint32_t*>(chunk)[lane] : 0u;
  const uint64_t nw = len > 128 ? (len - 128) / 2 : 0;
  const uint16_t* words = reinterpret_cast<const uint16_t*>(chunk + 128);
  const uint64_t base = from + k * kLLChunk;
  const uint32_t n = (uint32_t)min((uint64_t)kLLChunk, raw_total - base);
  const uint32_t below = (1u << lane) - 1u;
  // the words are taken in order, at most 32 per step: a window of 128 of them in registers
  // (lane l holds words wb + l, wb + 32 + l, ...), the last two groups loaded ahead of use
  auto word = [&](uint64_t q) -> uint32_t { return q < nw ? (uint32_t)words[q] : 0u; };
  uint64_t wb = 0, p = 0;
  uint32_t w0 = word(lane), w1 = word(32 + lane), w2 = word(64 + lane), w3 = word(96 + lane);
  for (uint32_t t = 0; t < (n + 31) / 32; ++t) {
    const uint32_t i = t * 32 + lane;
    const bool act = i < n;
    bool need = false;
    if (act) {
      const uint32_t slot = x & (kLLM - 1);
      const uint32_t b = sym[slot];
      raw[base + i] = (uint8_t)b;
      x = (cum[b + 1] - cum[b]) * (x >> kLLScale) + slot - cum[b];
      need = x < kRansLow;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    const uint32_t src = (uint32_t)(p - wb) + __popc(mask & below);  // < 64
    const uint32_t a = __shfl_sync(0xffffffffu, w0, src & 31), bw = __shfl_sync(0xffffffffu, w1, src & 31);
    if (need) x = (x << 16) | (src < 32 ? a : bw);
    p += __popc(mask);
    if (p - wb >= 32) {  // warp-uniform
      wb += 32;
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = word(wb + 96 + lane);
    }
  }
}

}  // namespace

void launch_ll_pack(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L) {
  // the chunk count is known on the device only; grids cover the most the scratch can hold
  const uint64_t max_chunks = (w.raw_cap + kLLChunk - 1) / kLLChunk;
  if (cudaMemsetAsync(w.llhist, 0, 256 * sizeof(unsigned long long), L.stream) != cudaSuccess) return;
  k_ll_hist<<<(unsigned)(2 * L.sms), 256, 0, L.stream>>>(w.raw, w.st, w.llhist);
  note_launch();
  k_ll_freq<<<1, 32, 0, L.stream>>>(w.st, w.llhist, out, w.llcum);
  note_launch();
  const unsigned chunk_ctas = (unsigned)std::max<uint64_t>(1, (max_chunks + 7) / 8);
  k_ll_encode<<<chunk_ctas, 256, 0, L.stream>>>(w.raw, w.st, w);
  note_launch();
  k_ll_scan<<<1, 1024, 0, L.stream>>>(w.st, w, out, cap);
  note_launch();
  k_ll_place<<<chunk_ctas + (unsigned)L.sms, 256, 0, L.stream>>>(w.st, w, out, chunk_ctas);
  note_launch();
  (void)g;
}

void launch_ll_unpack(const uint8_t* s, uint64_t nbytes, const Hdr& h, uint8_t* raw, State* st, const Launch& L) {
  const uint64_t nch = ll_chunks(h.L.sumdc, h.raw_total);
  const unsigned chunk_ctas = (unsigned)std::max<uint64_t>(1, (nch + 7) / 8);
  k_ll_unpack<<<chunk_ctas + (unsigned)L.sms, 256, 0, L.stream>>>(s, nbytes, h.L.sumdc, h.raw_total, raw, st,
                                                                  chunk_ctas);
  note_launch();
}

}  // namespace sdcsz
