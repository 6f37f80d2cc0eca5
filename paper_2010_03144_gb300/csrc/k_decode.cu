// K5: fault-tolerant decompression (Alg. 2 of the paper, without the Zstd stage).
//
// Persistent CTAs, each taking whole random-access groups of 256 blocks; one thread per
// block. A CTA builds a 12-bit first-level decode table for the canonical Huffman code in
// shared memory (longer codes resolve through the canonical first-code table), scans the
// group's block table for per-block offsets, checks the group table against it, and then each
// thread decodes its block and reconstructs it with the Lorenzo or regression predictor
// (lines 2-9). For fault-tolerant streams the block's checksum is compared with sum_dc
// (lines 11-13); on a mismatch the block is decompressed once more from its compressed bytes
// (line 14) and reported corrected (line 17) or as an SDC (line 19).
#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

struct Canon {
  uint32_t fc[kMaxLen + 2];  // first code of each length
  uint32_t fi[kMaxLen + 2];  // canonical index of that first code
  uint32_t nc[kMaxLen + 2];  // codes of each length
};

// MSB-first bit reader over one block's payload bytes.
struct BitReader {
  const uint8_t* p;
  const uint8_t* lim;  // end of the stream: never read at or past it
  unsigned long long buf;
  int nb;
  uint32_t used, total;
  __device__ __forceinline__ void refill() {
    while (nb <= 56) {
      const uint32_t byte = (p < lim) ? (uint32_t)*p : 0u;
      ++p;
      buf |= (unsigned long long)byte << (56 - nb);
      nb += 8;
    }
  }
  // returns the symbol, or -1 for an invalid code or when the block's bits run out
  __device__ __forceinline__ int next(const uint32_t* lut, const Canon& cn, const uint16_t* syms, uint32_t n_live) {
    if (nb < kMaxLen) refill();
    uint32_t e = lut[buf >> (64 - kLutBits)];
    uint32_t len, sym;
    if (e & 0xffu) {
      len = e & 0xffu;
      sym = e >> 8;
    } else {
      len = 0;
      sym = 0;
      for (uint32_t l = kLutBits + 1; l <= (uint32_t)kMaxLen; ++l) {
        const uint32_t c = (uint32_t)(buf >> (64 - l));
        if (c - cn.fc[l] < cn.nc[l]) {
          const uint32_t r = cn.fi[l] + (c - cn.fc[l]);
          if (r >= n_live) return -1;
          sym = syms[r];
          len = l;
          break;
        }
      }
      if (!len) return -1;
    }
    used += len;
    if (used > total) return -1;
    buf <<= len;
    nb -= (int)len;
    return (int)sym;
  }
};

struct BlockIn {
  uint64_t b, pay_off, un_off;
  uint32_t size, ucnt;
  int64_t reg_idx;
};

template <typename T, int NDIM>
__device__ bool decode_block(const uint8_t* __restrict__ s, const uint8_t* lim, const Hdr& h, const BlockIn& bi,
                             const uint32_t* lut, const Canon& cn, const uint16_t* syms, Walker<T, NDIM>& wk,
                             T* __restrict__ field, const T* __restrict__ orig, uint32_t kinj, uint32_t bitinj,
                             unsigned long long* sum_out, unsigned long long* viol, double* maxerr) {
  const Geo& g = h.g;
  const Box x = block_box(g, bi.b);
  const T eb = (T)h.eb;
  T cT[4] = {T(0), T(0), T(0), T(0)};
  const bool reg = bi.reg_idx >= 0;
  if (reg) {
    const T* c = reinterpret_cast<const T*>(s + h.L.coef) + (uint64_t)(NDIM + 1) * bi.reg_idx;
    for (int a = 0; a <= NDIM; ++a) cT[a] = c[a];
  }
  const T* un = reinterpret_cast<const T*>(s + h.L.unpred) + bi.un_off;
  BitReader br;
  br.p = s + h.L.payload + bi.pay_off;
  br.lim = lim;
  br.buf = 0;
  br.nb = 0;
  br.used = 0;
  br.total = bi.size * 8u;
  bool ok = true;
  uint32_t used_u = 0, k = 0;
  unsigned long long sum = 0, nv = 0;
  double me = 0.0;
  for (uint32_t i = 0; i < x.e[0]; ++i) {
    for (uint32_t j = 0; j < x.e[1]; ++j) {
      const uint64_t rb = row_base(g, x, i, j);
      wk.row_start();
      for (uint32_t l = 0; l < x.e[2]; ++l, ++k) {
        const int q = ok ? br.next(lut, cn, syms, h.n_live) : -1;
        T xr = T(0);
        if (!reg) wk.load(i, j, l);
        if (q < 0 || (uint32_t)q >= g.bins) {
          ok = false;
        } else if (q == 0) {
          if (used_u < bi.ucnt) xr = un[used_u];
          else ok = false;
          ++used_u;
        } else {
          const T pred = reg ? regress<T, NDIM, OpRN<T>>(cT, i, j, l) : wk.template combine<OpRN<T>>();
          xr = FT<T>::add(pred, FT<T>::mul(FT<T>::fromi(2 * (q - (int)g.R)), eb));
        }
        if (k == kinj) xr = FT<T>::flip(xr, bitinj);
        if (!reg) wk.commit(j, l, xr);
        if (field) field[rb + l] = xr;
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
        add_sum<T>(xr, sum);
      }
    }
  }
  if (used_u != bi.ucnt) ok = false;
  *sum_out = sum;
  *viol = nv;
  *maxerr = me;
  return ok;
}

__device__ __forceinline__ unsigned long long ld_u64(const uint8_t* p) {
  return *reinterpret_cast<const unsigned long long*>(p);
}

}  // namespace

template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_decode(const uint8_t* __restrict__ s, uint64_t nbytes, Hdr h, T* field,
                                                uint8_t* status, const T* orig, State* st,
                                                const sdcsz_flip* __restrict__ flips, uint32_t nflips) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Canon cn;
  __shared__ uint32_t s_sz[kGroup], s_uc[kGroup], s_rg[kGroup];
  __shared__ unsigned long long s_off[kGroup][3];
  __shared__ unsigned long long s_wt[8][3];
  __shared__ int s_bad;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const Geo& g = h.g;
  uint32_t* lut = reinterpret_cast<uint32_t*>(smem);
  const uint16_t* syms = reinterpret_cast<const uint16_t*>(s + h.L.table + 4 * (kMaxLen + 1));
  const uint8_t* lim = s + nbytes;

  // canonical tables and the first-level decode table
  if (tid == 0) {
    const uint32_t* blc = reinterpret_cast<const uint32_t*>(s + h.L.table);
    unsigned long long kraft = 0, total = 0;
    uint32_t code = 0, idx = 0;
    int bad = blc[0] != 0;
    for (uint32_t l = 1; l <= (uint32_t)kMaxLen; ++l) {
      const uint32_t c = blc[l];
      code = (code + (l >= 2 ? cn.nc[l - 1] : 0u)) << 1;
      cn.fc[l] = code;
      cn.fi[l] = idx;
      cn.nc[l] = c;
      idx += c;
      kraft += (unsigned long long)c << (kMaxLen - l);
      total += c;
    }
    if (total != h.n_live || kraft > (1ull << kMaxLen)) bad = 1;
    s_bad = bad;
    if (bad) atomicOr(&st->error, ERR_FORMAT);
  }
  __syncthreads();
  if (s_bad) return;
  for (uint32_t e = tid; e < (1u << kLutBits); e += blockDim.x) {
    uint32_t v = 0;
    for (uint32_t l = 1; l <= (uint32_t)kLutBits; ++l) {
      const uint32_t c = e >> (kLutBits - l);
      if (c - cn.fc[l] < cn.nc[l]) {
        const uint32_t r = cn.fi[l] + (c - cn.fc[l]);
        const uint32_t sym = r < h.n_live ? syms[r] : 0u;
        v = (sym << 8) | l;
        break;
      }
    }
    lut[e] = v;
  }

  Walker<T, NDIM> wk;
  wk.base = reinterpret_cast<T*>(smem + (4u << kLutBits)) + tid;
  wk.stride = blockDim.x;
  wk.B2 = g.B[2];
  wk.sr = g.B[1] * g.B[2];
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  unsigned long long c_fix = 0, c_bad = 0, c_viol = 0;
  double c_maxerr = 0.0;

  for (uint64_t gid = blockIdx.x; gid < ngroups; gid += gridDim.x) {
    __syncthreads();
    // the group's block table, scanned; thread t owns entries t, t + blockDim, ...
    const uint64_t b0 = gid * kGroup;
    const uint32_t nblk = (uint32_t)min((uint64_t)kGroup, g.nb - b0);
    for (uint32_t t = tid; t < kGroup; t += blockDim.x) {
      const uint64_t b = b0 + t;
      const bool in = t < nblk;
      s_sz[t] = in ? *reinterpret_cast<const uint16_t*>(s + h.L.sizes + 2 * b) : 0u;
      s_uc[t] = in ? *reinterpret_cast<const uint16_t*>(s + h.L.ucounts + 2 * b) : 0u;
      s_rg[t] = in ? ((*reinterpret_cast<const uint32_t*>(s + h.L.bitmap + 4 * (b / 32)) >> (b % 32)) & 1u) : 0u;
    }
    __syncthreads();
    {
      // thread t sums entries [t*R, t*R + R); warp scan of those sums; warp totals by thread 0
      const uint32_t R = kGroup / blockDim.x;
      unsigned long long loc[3] = {0, 0, 0};
      for (uint32_t r = 0; r < R; ++r) {
        const uint32_t e = tid * R + r;
        loc[0] += s_sz[e];
        loc[1] += s_uc[e];
        loc[2] += s_rg[e];
      }
      unsigned long long inc[3] = {loc[0], loc[1], loc[2]};
      for (int o = 1; o < 32; o <<= 1)
        for (int q = 0; q < 3; ++q) {
          const unsigned long long n = __shfl_up_sync(0xffffffffu, inc[q], o);
          if (lane >= (uint32_t)o) inc[q] += n;
        }
      if (lane == 31)
        for (int q = 0; q < 3; ++q) s_wt[wid][q] = inc[q];
      __syncthreads();
      if (tid == 0) {
        unsigned long long run[3] = {0, 0, 0};
        for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2)
          for (int q = 0; q < 3; ++q) {
            const unsigned long long t = s_wt[w2][q];
            s_wt[w2][q] = run[q];
            run[q] += t;
          }
        // the stored group bases must agree with the block table
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
        s_bad = bad;
        if (bad) atomicOr(&st->error, ERR_FORMAT);
        for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2)
          for (int q = 0; q < 3; ++q) s_wt[w2][q] += base[q];
      }
      __syncthreads();
      unsigned long long run[3];
      for (int q = 0; q < 3; ++q) run[q] = s_wt[wid][q] + inc[q] - loc[q];
      for (uint32_t r = 0; r < R; ++r) {
        const uint32_t e = tid * R + r;
        s_off[e][0] = run[0];
        s_off[e][1] = run[1];
        s_off[e][2] = run[2];
        run[0] += s_sz[e];
        run[1] += s_uc[e];
        run[2] += s_rg[e];
      }
    }
    __syncthreads();
    if (s_bad) {
      if (status)
        for (uint32_t t = tid; t < nblk; t += blockDim.x) status[b0 + t] = SDCSZ_BLOCK_BAD;
      continue;
    }

    for (uint32_t t = tid; t < nblk; t += blockDim.x) {
      BlockIn bi;
      bi.b = b0 + t;
      bi.pay_off = s_off[t][0];
      bi.un_off = s_off[t][1];
      bi.reg_idx = s_rg[t] ? (int64_t)s_off[t][2] : -1;
      bi.size = s_sz[t];
      bi.ucnt = s_uc[t];
      uint32_t kinj = 0xffffffffu, bitinj = 0;
      if (nflips) {
        uint64_t idx;
        uint32_t bit;
        if (find_flip(flips, nflips, SDCSZ_SITE_DECOMP, bi.b, &idx, &bit)) {
          kinj = (uint32_t)idx;
          bitinj = bit;
        }
      }
      unsigned long long sum = 0, nv = 0;
      double me = 0.0;
      bool ok = decode_block<T, NDIM>(s, lim, h, bi, lut, cn, syms, wk, field, orig, kinj, bitinj, &sum, &nv, &me);
      uint8_t stv = SDCSZ_BLOCK_OK;
      if (g.abft) {
        const unsigned long long ref = ld_u64(s + h.L.sumdc + 8 * bi.b);
        if (!ok || sum != ref) {
          // Alg. 2 line 14: decompress this block again from its compressed bytes
          ok = decode_block<T, NDIM>(s, lim, h, bi, lut, cn, syms, wk, field, orig, 0xffffffffu, 0, &sum, &nv, &me);
          if (ok && sum == ref) {
            stv = SDCSZ_BLOCK_CORRECTED;
            ++c_fix;
          } else {
            stv = ok ? SDCSZ_BLOCK_SDC : SDCSZ_BLOCK_BAD;
            ++c_bad;
          }
        }
      } else if (!ok) {
        stv = SDCSZ_BLOCK_BAD;
        ++c_bad;
      }
      c_viol += nv;
      c_maxerr = fmax(c_maxerr, me);
      if (status) status[bi.b] = stv;
    }
  }
  c_fix = warp_sum(c_fix);
  c_bad = warp_sum(c_bad);
  c_viol = warp_sum(c_viol);
  for (int o = 16; o > 0; o >>= 1) c_maxerr = fmax(c_maxerr, __shfl_xor_sync(0xffffffffu, c_maxerr, o));
  if (lane == 0) {
    if (c_fix) atomicAdd(&st->reexec_corrected, c_fix);
    if (c_bad) atomicAdd(&st->uncorrectable, c_bad);
    if (c_viol) atomicAdd(&st->bound_viol, c_viol);
    if (c_maxerr > 0.0) atomicMax(&st->max_err_bits, (unsigned long long)__double_as_longlong(c_maxerr));
  }
}

template <typename T, int NDIM>
static void run_decode(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                       const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                       const Launch& L) {
  const size_t per = (size_t)walker_slots(h.g.ndim, h.g.B) * sizeof(T);
  uint32_t threads = 256;
  while (threads > 64 && per * threads > 192 * 1024) threads >>= 1;
  const size_t smem = (4u << kLutBits) + per * threads;
  auto kern = k_decode<T, NDIM>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (int)threads, smem);
  if (occ < 1) occ = 1;
  const uint64_t ngroups = (h.g.nb + kGroup - 1) / kGroup;
  const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(ngroups, (uint64_t)occ * L.sms));
  kern<<<(unsigned)grid, threads, smem, L.stream>>>(s, nbytes, h, write ? static_cast<T*>(field) : nullptr, status,
                                                    static_cast<const T*>(original), st, flips, nflips);
}

void launch_decode(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                   const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                   const Launch& L) {
  if (h.g.nb == 0) return;
  if (h.g.dtype == 0) {
    if (h.g.ndim == 3) run_decode<float, 3>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
    else if (h.g.ndim == 2) run_decode<float, 2>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
    else run_decode<float, 1>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
  } else {
    if (h.g.ndim == 3) run_decode<double, 3>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
    else if (h.g.ndim == 2) run_decode<double, 2>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
    else run_decode<double, 1>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
  }
}

}  // namespace sdcsz
