// K3: Huffman code for the whole bin array (Algorithm 1), the stream header and the
// section layout. One CTA of 1024 threads.
//
//   1. compact the live symbols into keys (count << 16 | symbol) and sort them ascending:
//      leaves in increasing (count, symbol) order;
//   2. two-queue Huffman merge (one thread): the next node is the lighter of the next leaf
//      and the oldest unmerged internal node, a leaf winning ties. This is Huffman's
//      algorithm with ties broken by creation order (leaves first, in sorted order);
//   3. leaf depths, then lengths longer than 24 bits are reduced by the JPEG adjustment
//      (ITU-T T.81 Annex K.3) and handed out longest-first to the leaves in sorted order;
//   4. canonical codes: symbols sorted by (length, symbol) get consecutive codes per length.
#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

constexpr uint32_t kSmemSort = 8192;  // keys sorted in shared memory up to this many
constexpr size_t kCodebookMerge = 224 * 1024;  // the kernels' dynamic shared memory
static_assert(kCodebookMerge >= kSmemSort * 8 + 8192 * 4 + 16384 * 4, "the small case's arrays fit");

// Ascending bitonic sort of n_pad (power of two) 64-bit keys, shared or global memory.
__device__ void bitonic_sort(unsigned long long* a, uint32_t n_pad) {
  for (uint32_t size = 2; size <= n_pad; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t t = threadIdx.x; t < n_pad / 2; t += blockDim.x) {
        const uint32_t i = 2 * t - (t & (stride - 1));
        const uint32_t j = i + stride;
        const bool up = (i & size) == 0;
        const unsigned long long x = a[i], y = a[j];
        if ((x > y) == up) {
          a[i] = y;
          a[j] = x;
        }
      }
      __syncthreads();
    }
  }
}

// Ascending sort of n distinct keys (padded to n_pad with ~0). Up to one key per thread: each
// thread counts the keys below its own (all threads read the same key at a time, a broadcast)
// and stores it at that rank; three barriers instead of the bitonic network's many.
__device__ void sort_global(unsigned long long* a, unsigned long long* tmp, uint32_t n_pad, unsigned long long* s);

// (tmp, s: scratch of sort_global for n_pad above kSmemSort)
__device__ void sort_keys(unsigned long long* a, uint32_t n, uint32_t n_pad, unsigned long long* tmp = nullptr,
                          unsigned long long* s = nullptr) {
  if (n <= 1) return;
  if (n_pad > kSmemSort) {
    sort_global(a, tmp, n_pad, s);
    return;
  }
  if (n > blockDim.x) {
    bitonic_sort(a, n_pad);
    return;
  }
  const uint32_t t = threadIdx.x;
  unsigned long long mine = 0;
  uint32_t rank = 0;
  __syncthreads();
  if (t < n) {
    mine = a[t];
    for (uint32_t j = 0; j < n; ++j) rank += a[j] < mine;
  }
  __syncthreads();
  if (t < n) a[rank] = mine;
  __syncthreads();
}

__device__ __forceinline__ void put_u8(uint8_t* o, uint64_t off, uint8_t v) { o[off] = v; }
__device__ __forceinline__ void put_u16(uint8_t* o, uint64_t off, uint16_t v) {
  o[off] = (uint8_t)v; o[off + 1] = (uint8_t)(v >> 8);
}
__device__ __forceinline__ void put_u32(uint8_t* o, uint64_t off, uint32_t v) {
  for (int q = 0; q < 4; ++q) o[off + q] = (uint8_t)(v >> (8 * q));
}
__device__ __forceinline__ void put_u64(uint8_t* o, uint64_t off, unsigned long long v) {
  for (int q = 0; q < 8; ++q) o[off + q] = (uint8_t)(v >> (8 * q));
}

// Leaf weights for the merge: the counts of sorted keys (count << 16 | symbol), or a copy of
// them as 32-bit values.
struct KeyLeaf {
  const unsigned long long* __restrict__ k;
  __device__ __forceinline__ unsigned long long operator()(uint32_t i) const { return k[i] >> 16; }
};
struct U32Leaf {
  const uint32_t* __restrict__ v;
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return v[i]; }
};

// Ascending sort of n_pad (a power of two above kSmemSort) distinct keys in global memory:
// runs of kSmemSort keys sorted in shared memory (s), then merge rounds between a and tmp,
// each thread producing n_pad / blockDim.x consecutive outputs from where a binary search on
// its diagonal (the merge path) puts them. The result ends in a.
__device__ void sort_global(unsigned long long* a, unsigned long long* tmp, uint32_t n_pad, unsigned long long* s) {
  for (uint32_t base = 0; base < n_pad; base += kSmemSort) {
    for (uint32_t t = threadIdx.x; t < kSmemSort; t += blockDim.x) s[t] = a[base + t];
    __syncthreads();
    bitonic_sort(s, kSmemSort);
    for (uint32_t t = threadIdx.x; t < kSmemSort; t += blockDim.x) a[base + t] = s[t];
    __syncthreads();
  }
  unsigned long long *src = a, *dst = tmp;
  const uint32_t per = n_pad / blockDim.x;
  for (uint32_t wdt = kSmemSort; wdt < n_pad; wdt <<= 1) {
    const uint32_t o0 = threadIdx.x * per;
    const uint32_t base = o0 / (2 * wdt) * (2 * wdt), d = o0 - base;
    const unsigned long long* A = src + base;
    const unsigned long long* Bk = src + base + wdt;
    uint32_t lo = d > wdt ? d - wdt : 0, hi = d < wdt ? d : wdt;
    while (lo < hi) {  // the number of A's keys among the pair's d smallest
      const uint32_t mid = (lo + hi) >> 1;
      if (A[mid] < Bk[d - 1 - mid]) lo = mid + 1;
      else hi = mid;
    }
    uint32_t i = lo, j = d - lo;
    for (uint32_t q = 0; q < per; ++q) {
      const bool takeA = i < wdt && (j >= wdt || A[i] < Bk[j]);
      dst[base + d + q] = takeA ? A[i] : Bk[j];
      i += takeA ? 1u : 0u;
      j += takeA ? 0u : 1u;
    }
    __syncthreads();
    unsigned long long* t = src;
    src = dst;
    dst = t;
  }
  if (src != a) {
    for (uint32_t t = threadIdx.x; t < n_pad; t += blockDim.x) a[t] = src[t];
    __syncthreads();
  }
}

// Huffman's algorithm on n >= 2 leaves sorted by (count, symbol), with two queues: the next node
// is the lighter of the next leaf and the oldest unmerged internal node, a leaf winning ties
// (ties broken by creation order, leaves first in sorted order). Writes every node's parent
// (leaves 0..n-1, internal nodes n..2n-2). W holds any weight (a sum of counts).
// One thread; the next two leaf weights and the next two internal weights are kept in
// registers, so a pick compares registers, and the loads that refill them are issued a pick
// or more before their values are needed; a node just created is forwarded.
template <typename W, class Leaf>
__device__ __forceinline__ void huffman_merge(Leaf leafw, uint32_t n, W* __restrict__ iw, uint32_t* __restrict__ parent) {
  uint32_t lp = 0, ip = 0;
  W l0 = (W)leafw(0), l1 = (W)leafw(1), h0 = 0, h1 = 0;
  for (uint32_t ni = 0; ni + 1 < n; ++ni) {
    W wsum = 0;
#pragma unroll
    for (int pick = 0; pick < 2; ++pick) {
      // internal nodes waiting: ni - ip (h0 is the oldest, h1 the next when there are two);
      // both refills are loaded (from clamped addresses) and the pick selects, without a branch
      const bool leaf = lp < n && (ip >= ni || l0 <= h0);
      const W nl = (W)leafw(min(lp + 2, n - 1));
      const W nh = iw[ip + 2 < ni ? ip + 2 : 0];
      wsum += leaf ? l0 : h0;
      parent[leaf ? lp : n + ip] = n + ni;
      l0 = leaf ? l1 : l0;
      l1 = leaf ? nl : l1;
      h0 = leaf ? h0 : h1;
      h1 = leaf ? h1 : nh;
      lp += leaf ? 1u : 0u;
      ip += leaf ? 0u : 1u;
    }
    iw[ni] = wsum;
    if (ip == ni) h0 = wsum;            // the only waiting node is the one just made
    else if (ip + 1 == ni) h1 = wsum;   // it is the second in line
  }
}

}  // namespace

__device__ __forceinline__ void codebook(const Geo& g, const Ws& w, uint8_t* __restrict__ out, uint64_t cap,
                                         unsigned char* smem) {
  __shared__ uint32_t cnt[64];
  __shared__ uint32_t s_maxlen;
  __shared__ uint32_t first_code[kMaxLen + 2], first_index[kMaxLen + 2], cum[kMaxLen + 2];
  State* st = w.st;
  const uint32_t tid = threadIdx.x;

  // 1. the live symbols' keys (count << 16 | symbol), gathered by k_codebook_gather in no
  //    particular order (they are sorted next) together with their number
  const uint32_t n = *(volatile unsigned int*)&st->n_live;
  uint32_t n_pad = 1;
  while (n_pad < n) n_pad <<= 1;
  unsigned long long* keys = (n_pad <= kSmemSort) ? reinterpret_cast<unsigned long long*>(smem) : w.sort_keys;
  __syncthreads();
  for (uint32_t t = tid; t < n_pad; t += blockDim.x) keys[t] = (t < n) ? w.sort_keys[t] : ~0ull;
  __syncthreads();
  sort_keys(keys, n, n_pad, w.node_w, reinterpret_cast<unsigned long long*>(smem));
  for (uint32_t t = tid; t < 64; t += blockDim.x) cnt[t] = 0;
  if (tid == 0) s_maxlen = 0;
  __syncthreads();

  // 2-3. Huffman merge and leaf depths (one thread), length counts
  if (n >= 2) {
    // node arrays: internal weights [n-1], parents [2n-1]; in shared memory when they fit
    // (32-bit weights, used when the field has fewer than 2^32 points, fit twice as many)
    const bool w32 = g.N < (1ull << 32);
    const bool small = n <= (w32 ? 8192u : 4096u);  // then the keys are in shared memory too
    // more leaves (keys in global memory): 32-bit copies of the leaf weights and the internal
    // weights in the shared memory the keys did not need, the parents in global memory
    const bool mid = !small && w32 && 8ull * n <= kCodebookMerge;
    uint32_t* parent = small ? reinterpret_cast<uint32_t*>(smem + kSmemSort * 8 + 8192 * 4) : w.node_parent;
    if (mid) {
      uint32_t* lws = reinterpret_cast<uint32_t*>(smem);
      for (uint32_t t = tid; t < n; t += blockDim.x) lws[t] = (uint32_t)(keys[t] >> 16);
      __syncthreads();
    }
    if (tid == 0) {
      if (small) {  // every array in shared memory (addresses the compiler sees as shared)
        const KeyLeaf ks{reinterpret_cast<const unsigned long long*>(smem)};
        uint32_t* ps = reinterpret_cast<uint32_t*>(smem + kSmemSort * 8 + 8192 * 4);
        if (w32) huffman_merge<uint32_t>(ks, n, reinterpret_cast<uint32_t*>(smem + kSmemSort * 8), ps);
        else huffman_merge<unsigned long long>(ks, n, reinterpret_cast<unsigned long long*>(smem + kSmemSort * 8), ps);
      } else if (mid) {
        const U32Leaf ls{reinterpret_cast<const uint32_t*>(smem)};
        huffman_merge<uint32_t>(ls, n, reinterpret_cast<uint32_t*>(smem) + n, w.node_parent);
      } else if (w32) {
        huffman_merge<uint32_t>(KeyLeaf{keys}, n, reinterpret_cast<uint32_t*>(w.node_w), w.node_parent);
      } else {
        huffman_merge<unsigned long long>(KeyLeaf{keys}, n, w.node_w, w.node_parent);
      }
    }
    __syncthreads();
    // leaf depths: every leaf walks to the root (a Huffman tree over at most 2^40 points is
    // less than 64 levels deep) and counts its length
    {
      const uint32_t root = 2 * n - 2;
      for (uint32_t p = tid; p < n; p += blockDim.x) {
        uint32_t d = 0, v = p;
        while (v != root && d < 2 * n) {
          v = parent[v];
          ++d;
        }
        const uint32_t dc = d > 63 ? 63u : d;
        atomicAdd(&cnt[dc], 1u);
        atomicMax(&s_maxlen, dc);
      }
    }
    __syncthreads();
    if (tid == 0) {
      // JPEG Annex K.3: move pairs of the deepest codes up until none is longer than 24 bits
      for (uint32_t l = s_maxlen; l > (uint32_t)kMaxLen; --l) {
        while (cnt[l] > 0) {
          uint32_t j = l - 2;
          while (cnt[j] == 0) --j;
          cnt[l] -= 2;
          cnt[l - 1] += 1;
          cnt[j + 1] += 2;
          cnt[j] -= 1;
        }
      }
      // cum[l] = number of leaves with length > l (longest first)
      uint32_t acc = 0;
      for (int l = kMaxLen; l >= 0; --l) {
        cum[l] = acc;
        acc += cnt[l];
      }
      cum[kMaxLen + 1] = 0;
    }
  } else if (n == 1) {
    if (tid == 0) {
      cnt[1] = 1;
      cum[1] = 0;
      cum[0] = 1;
      for (int l = 2; l <= kMaxLen + 1; ++l) cum[l] = 0;
    }
  }
  __syncthreads();

  // lengths by leaf rank, then re-sort by (length, symbol) for the canonical order
  for (uint32_t p = tid; p < n; p += blockDim.x) {
    uint32_t len = 1;
    for (uint32_t l = 1; l <= (uint32_t)kMaxLen; ++l)
      if (cnt[l] && p >= cum[l] && p < cum[l] + cnt[l]) len = l;
    const unsigned long long sym = keys[p] & 0xffffull;
    w.sort_keys[p] = ((unsigned long long)len << 16) | sym;  // stage in global: keys may alias
  }
  __syncthreads();
  for (uint32_t t = tid; t < n_pad; t += blockDim.x) keys[t] = (t < n) ? w.sort_keys[t] : ~0ull;
  __syncthreads();
  sort_keys(keys, n, n_pad, w.node_w, reinterpret_cast<unsigned long long*>(smem));
  if (tid == 0) {
    uint32_t code = 0, idx = 0;
    for (uint32_t l = 1; l <= (uint32_t)kMaxLen; ++l) {
      code = (code + (l >= 2 ? cnt[l - 1] : 0u)) << 1;
      first_code[l] = code;
      first_index[l] = idx;
      idx += cnt[l];
    }
  }
  __syncthreads();

  // the stream layout now that every section size is known
  const Layout L = make_layout(g, n, st->n_reg, st->n_unpred);
  if (L.payload > cap) {
    if (tid == 0) atomicOr(&st->error, ERR_CAPACITY);
    return;
  }
  for (uint32_t r = tid; r < n; r += blockDim.x) {
    const uint32_t len = (uint32_t)(keys[r] >> 16);
    const uint32_t sym = (uint32_t)(keys[r] & 0xffffu);
    const uint32_t code = first_code[len] + (r - first_index[len]);
    w.codebook[sym] = (code << 5) | len;
    if (out) put_u16(out, L.table + 4 * (kMaxLen + 1) + 2 * (uint64_t)r, (uint16_t)sym);
  }
  if (out && tid <= (uint32_t)kMaxLen) put_u32(out, L.table + 4 * tid, tid == 0 ? 0u : cnt[tid]);
  if (tid == 0) {
    st->n_live = n;
    st->L = L;
    st->payload_bytes = 0;
    st->total_bytes = L.payload;
  }
  // no output: the codebook and the layout only (a shard of a field whose header another writes)
  if (tid == 0 && out) {
    // header (128 bytes, little-endian)
    for (int q = 0; q < kHeaderBytes; ++q) out[q] = 0;
    out[0] = 'S'; out[1] = 'D'; out[2] = 'S'; out[3] = 'Z';
    put_u16(out, 4, 1);
    put_u8(out, 6, (uint8_t)g.dtype);
    put_u8(out, 7, (uint8_t)g.ndim);
    const int off = 3 - g.ndim;
    for (int a = 0; a < g.ndim; ++a) {
      put_u64(out, 8 + 8 * a, g.d[off + a]);
      put_u32(out, 32 + 4 * a, g.B[off + a]);
    }
    put_u32(out, 44, g.bins);
    put_u8(out, 48, (uint8_t)g.abft);
    put_u8(out, 49, (uint8_t)g.predictor);
    put_u8(out, 50, (uint8_t)g.eb_mode);
    put_u8(out, 51, (uint8_t)g.enc);
    put_u32(out, 52, n);
    put_u64(out, 56, (unsigned long long)__double_as_longlong(st->eb));
    put_u64(out, 64, (unsigned long long)__double_as_longlong(g.e));
    put_u64(out, 72, g.nb);
    put_u64(out, 80, st->n_reg);
    put_u64(out, 88, st->n_unpred);
    put_u64(out, 96, 0);
    put_u64(out, 104, L.payload);
    put_u32(out, 112, st->uncorrectable ? 1u : 0u);
    // zero the alignment gaps between sections
    const uint64_t s = g.dtype ? 8 : 4;
    const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
    const uint64_t ends[8] = {L.table + 4 * (kMaxLen + 1) + 2 * (uint64_t)n, L.groups + 24 * ngroups,
                              L.sizes + 2 * g.nb, L.ucounts + 2 * g.nb, L.bitmap + 4 * ((g.nb + 31) / 32),
                              L.sumdc + (g.abft ? 8 * g.nb : 0),
                              L.coef + (g.enc ? 0 : s * (uint64_t)(g.ndim + 1) * st->n_reg),
                              L.unpred + (g.enc ? 0 : s * st->n_unpred)};
    const uint64_t starts[8] = {L.groups, L.sizes, L.ucounts, L.bitmap, L.sumdc, L.coef, L.unpred, L.payload};
    for (int q = 0; q < 8; ++q)
      for (uint64_t o = ends[q]; o < starts[q]; ++o) out[o] = 0;
    // the last bitmap word may be partial: it is written whole by the encoder
  }
}

// Step 1 of the codebook, spread over the GPU: one thread per bin clears the codebook entry and,
// for a live bin, appends its key (warp-aggregated slot reservation on State::n_live).
__device__ __forceinline__ void gather_bin(const Geo& g, const Ws& w, uint32_t s) {
  const uint32_t lane = threadIdx.x & 31;
  const unsigned long long hc = s < g.bins ? __ldg(&w.hist[s]) : 0ull;
  if (s < g.bins) w.codebook[s] = 0;
  const unsigned int m = __ballot_sync(0xffffffffu, hc != 0);
  uint32_t base = 0;
  if (lane == 0 && m) base = atomicAdd(&w.st->n_live, (unsigned int)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (hc) w.sort_keys[base + __popc(m & ((1u << lane) - 1))] = (hc << 16) | s;
}

__global__ void __launch_bounds__(1024) k_codebook_gather(Geo g, Ws w) {
  gather_bin(g, w, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(1024) k_codebook_gather_batch(const Job* __restrict__ jobs) {
  const Job& jb = jobs[blockIdx.y];
  gather_bin(jb.g, jb.w, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(1024) k_codebook(Geo g, Ws w, uint8_t* __restrict__ out, uint64_t cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (*(volatile unsigned int*)&w.st->error) return;
  codebook(g, w, out, cap, smem);
}

// One CTA per job of a batch.
__global__ void __launch_bounds__(1024) k_codebook_batch(const Job* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Job s_job;
  __shared__ int s_skip;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&jobs[blockIdx.x]);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_job);
  for (uint32_t q = threadIdx.x; q < sizeof(Job) / 8; q += blockDim.x) dst[q] = src[q];
  __syncthreads();
  if (threadIdx.x == 0) s_skip = *(volatile unsigned int*)&s_job.w.st->error != 0;
  __syncthreads();
  if (s_skip) return;
  codebook(s_job.g, s_job.w, s_job.out, s_job.cap, smem);
}

// keys (kSmemSort x 8), internal weights (8192 x 4, or 4096 x 8), parents (16384 x 4); for more
// leaves, their 32-bit weights and the internal weights (kCodebookMerge bytes: 28672 leaves)
constexpr size_t kCodebookSmem = kCodebookMerge;

void batch_codebook(const Job* jobs, uint32_t n, const Launch& L) {
  k_codebook_gather_batch<<<dim3(64, n), 1024, 0, L.stream>>>(jobs);
  note_launch();
  allow_smem(reinterpret_cast<const void*>(k_codebook_batch), kCodebookSmem);
  k_codebook_batch<<<n, 1024, kCodebookSmem, L.stream>>>(jobs);
  note_launch();
}

void launch_codebook(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L) {
  const size_t smem = kCodebookSmem;
  k_codebook_gather<<<(g.bins + 1023) / 1024, 1024, 0, L.stream>>>(g, w);
  note_launch();
  allow_smem(reinterpret_cast<const void*>(k_codebook), smem);
  k_codebook<<<1, 1024, smem, L.stream>>>(g, w, out, cap);
  note_launch();
}

}  // namespace sdcsz
