// K4: per-block Huffman encoding and stream assembly (Alg. 1 lines 34-40 of the paper,
// without the Zstd stage).
//
// One CTA per random-access group of 256 blocks, one thread per block. Pass 1 reads the
// block's codes, checks them against sum_q/isum_q (line 35: a single corrupted code is located
// and repaired) and sums the code lengths. A CTA scan plus a single-pass decoupled look-back
// across groups (group ids taken from a ticket in launch order, every wait bounded) gives each
// block its payload, unpredictable-value and coefficient offsets. Pass 2 re-reads the codes
// (L2 resident), packs the bits MSB-first and writes the block table entries.
#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

constexpr unsigned long long kFlagAgg = 1ull, kMaskBytes = (1ull << 22) - 1, kMaskUn = (1ull << 21) - 1;

__device__ __forceinline__ unsigned long long pack_agg(unsigned long long bytes, unsigned long long un,
                                                       unsigned long long rg) {
  return (kFlagAgg << 62) | (rg << 43) | (un << 22) | bytes;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(256) k_encode(Geo g, Ws w, uint8_t* __restrict__ out, uint64_t cap) {
  __shared__ uint32_t s_gid;
  __shared__ unsigned long long s_wt[8][3];
  __shared__ unsigned long long s_excl[3];
  __shared__ unsigned long long s_tot[3];
  State* st = w.st;
  if (*(volatile unsigned int*)&st->error) return;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_gid = atomicAdd(&st->ticket, 1u);
  __syncthreads();
  const uint64_t gid = s_gid;
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  const uint64_t b = gid * kGroup + tid;
  const bool active = b < g.nb;
  const Layout L = st->L;

  // pass 1: verify codes, count bits and unpredictables
  Box x;
  x.P = 0;
  uint32_t bits = 0, nun = 0, kfix = 0xffffffffu, vfix = 0;
  bool reg = false, bad = false;
  if (active) {
    x = block_box(g, b);
    reg = w.flags[b] & 1;
    unsigned long long s = 0, is = 0;
    uint64_t ci = code_index(b, g.P, 0);
    for (uint32_t k = 0; k < x.P; ++k, ci += 32) {
      const uint32_t c = w.codes[ci];
      bits += __ldg(&w.codebook[c]) & 31u;
      nun += (c == 0);
      s += c;
      is += (unsigned long long)(k + 1) * c;
    }
    if (g.abft && (s != w.sum_q[b] || is != w.isum_q[b])) {
      long long delta = 0;
      const long long m = locate_word(w.sum_q[b], w.isum_q[b], s, is, x.P, 0, &delta);
      bool fixed = false;
      if (m >= 0) {
        const uint32_t old = w.codes[code_index(b, g.P, (uint32_t)m)];
        const long long nv = (long long)old - delta;
        if (nv >= 0 && nv < (long long)g.bins) {
          kfix = (uint32_t)m;
          vfix = (uint32_t)nv;
          bits += (__ldg(&w.codebook[vfix]) & 31u) - (__ldg(&w.codebook[old]) & 31u);
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
  if (tid == 0) {
    unsigned long long run[3] = {0, 0, 0};
    for (int q2 = 0; q2 < 8; ++q2)
      for (int q = 0; q < 3; ++q) {
        unsigned long long t = s_wt[q2][q];
        s_wt[q2][q] = run[q];
        run[q] += t;
      }
    for (int q = 0; q < 3; ++q) s_tot[q] = run[q];
    // decoupled look-back: publish the aggregate, sum predecessors until an inclusive prefix
    LookBack* me = &w.lb[gid];
    unsigned long long excl[3] = {0, 0, 0};
    if (gid == 0) {
      me->incl[0] = run[0];
      me->incl[1] = run[1];
      me->incl[2] = run[2];
      __threadfence();
      *(volatile unsigned int*)&me->incl_flag = 1u;
    } else {
      *(volatile unsigned long long*)&me->agg = pack_agg(run[0], run[1], run[2]);
      __threadfence();
      int64_t p = (int64_t)gid - 1;
      while (p >= 0) {
        const LookBack* pr = &w.lb[p];
        uint32_t spins = 0;
        bool done = false;
        for (;;) {
          if (*(volatile const unsigned int*)&pr->incl_flag) {
            __threadfence();
            excl[0] += *(volatile const unsigned long long*)&pr->incl[0];
            excl[1] += *(volatile const unsigned long long*)&pr->incl[1];
            excl[2] += *(volatile const unsigned long long*)&pr->incl[2];
            done = true;
            break;
          }
          const unsigned long long a = ld_volatile(&pr->agg);
          if (a >> 62) {
            excl[0] += a & kMaskBytes;
            excl[1] += (a >> 22) & kMaskUn;
            excl[2] += (a >> 43) & 0x7ffffull;
            break;
          }
          if (++spins > kSpinLimit) {
            atomicOr(&st->error, ERR_TIMEOUT);
            done = true;
            break;
          }
          __nanosleep(64);
        }
        if (done) break;
        --p;
      }
      me->incl[0] = excl[0] + run[0];
      me->incl[1] = excl[1] + run[1];
      me->incl[2] = excl[2] + run[2];
      __threadfence();
      *(volatile unsigned int*)&me->incl_flag = 1u;
    }
    for (int q = 0; q < 3; ++q) s_excl[q] = excl[q];
  }
  __syncthreads();

  const uint64_t s_dt = g.dtype ? 8 : 4;
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
  if (g.abft) *reinterpret_cast<unsigned long long*>(out + L.sumdc + 8 * b) = w.sum_dc[b];
  if (reg) {
    const T* cT = static_cast<const T*>(w.coefT) + 4 * b;
    T* dst = reinterpret_cast<T*>(out + L.coef) + (uint64_t)(g.ndim + 1) * rg_off;
    for (int a = 0; a <= g.ndim; ++a) dst[a] = cT[a];
  }
  // pass 2: pack the codes MSB-first; copy the unpredictable values in order
  const uint64_t pstart = L.payload + pay_off;
  const bool fits = pstart + bytes <= cap;
  if (!fits) atomicOr(&st->error, ERR_CAPACITY);
  uint8_t* dst = out + pstart;
  const T* ust = static_cast<const T*>(w.ustage);
  T* udst = reinterpret_cast<T*>(out + L.unpred);
  unsigned long long uidx = un_off;
  const unsigned long long ulim = st->n_unpred;
  unsigned long long acc = 0;
  uint32_t nacc = 0;
  uint64_t ci = code_index(b, g.P, 0);
  for (uint32_t k = 0; k < x.P; ++k, ci += 32) {
    uint32_t c = w.codes[ci];
    if (k == kfix) c = vfix;
    const uint32_t cw = __ldg(&w.codebook[c]);
    const uint32_t len = cw & 31u;
    acc = (acc << len) | (cw >> 5);
    nacc += len;
    while (nacc >= 8) {
      nacc -= 8;
      if (fits) *dst = (uint8_t)(acc >> nacc);
      ++dst;
    }
    if (c == 0) {
      if (uidx < ulim) udst[uidx] = ust[ci];
      ++uidx;
    }
  }
  if (nacc && fits) *dst = (uint8_t)(acc << (8 - nacc));
  if (bad) {
    // a block whose codes could not be repaired is reported in the header status word
    atomicOr(reinterpret_cast<unsigned int*>(out + 112), 1u);
  }
  (void)s_dt;
}

void launch_encode(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L) {
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  if (!ngroups) return;
  if (g.dtype == 0) k_encode<float><<<(unsigned)ngroups, 256, 0, L.stream>>>(g, w, out, cap);
  else k_encode<double><<<(unsigned)ngroups, 256, 0, L.stream>>>(g, w, out, cap);
}

}  // namespace sdcsz
