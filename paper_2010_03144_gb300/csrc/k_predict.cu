// K2: prediction, quantization and block checksums (Alg. 1 lines 8 and 10-32 of the paper).
//
// One thread per block, a warp per 32 consecutive blocks, persistent CTAs. Per block:
//   * predictor choice from the K1 estimates (line 8),
//   * one pass over the block in its sequential order: prediction evaluated twice
//     (f_dup, line 18), linear-scaling quantization (lines 19-21), reconstruction evaluated
//     twice (dec_dup, line 25), the machine-epsilon double check (lines 26-28), the code,
//     sum_q/isum_q (line 24) and sum_dc (line 29), and the input words' checksums;
//   * the input check of line 11 is done speculatively: the words used by the pass are
//     summed on the fly and compared with sum_in/isum_in at the end; a mismatch (a memory
//     error since K1) is located, repaired, and the block is run again with the repaired
//     value, so the output equals that of an error-free run.
// Codes and unpredictable values go to warp-interleaved staging arrays (coalesced stores);
// the code histogram is privatised in shared memory around the central bin.
#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

struct PassRes {
  unsigned long long sw, isw;      // checksums of the input words used
  unsigned long long sq, isq, sdc; // sum_q, isum_q, sum_dc
  uint32_t nun, dup;
};

struct Hist {
  uint32_t* s;               // shared window
  unsigned long long* g;     // global histogram
  uint32_t lo, hi;
  __device__ __forceinline__ void add(uint32_t code, uint32_t cnt) const {
    if (code >= lo && code < hi) atomicAdd(&s[code - lo], cnt);
    else atomicAdd(&g[code], (unsigned long long)cnt);
  }
  __device__ __forceinline__ void sub1(uint32_t code) const {
    if (code >= lo && code < hi) atomicSub(&s[code - lo], 1u);
    else atomicAdd(&g[code], ~0ull);
  }
};

template <typename T, int NDIM, bool REG, bool ABFT>
__device__ __forceinline__ PassRes run_pass(const T* __restrict__ field, const Geo& g, const Box& x, uint64_t b,
                                            const T* cT, Walker<T, NDIM>& wk, T eb, T inv2, T Rh,
                                            uint16_t* __restrict__ codes, T* __restrict__ ustage, const Hist& h,
                                            uint32_t kp, uint32_t bitp, uint32_t kr, uint32_t bitr, uint32_t kfix,
                                            T xfix) {
  PassRes r = {0, 0, 0, 0, 0, 0, 0};
  uint32_t run_code = 0xffffffffu, run_len = 0;
  uint64_t ci = code_index(b, g.P, 0);
  uint32_t k = 0;
  const T half = T(0.5);
  for (uint32_t i = 0; i < x.e[0]; ++i) {
    for (uint32_t j = 0; j < x.e[1]; ++j) {
      const T* row = field + row_base(g, x, i, j);
      if (!REG) wk.row_start();
      for (uint32_t l = 0; l < x.e[2]; ++l, ++k, ci += 32) {
        const T v = (k == kfix) ? xfix : __ldg(row + l);
        if (ABFT) add_words<T>(v, k, r.sw, r.isw);
        // line 18: pred' <- f_dup(); a disagreement is settled by a third evaluation
        T pred;
        if (REG) {
          pred = regress<T, NDIM, OpRN<T>>(cT, i, j, l);
        } else {
          wk.load(i, j, l);
          pred = wk.template combine<OpRN<T>>();
        }
        if (ABFT) {
          if (k == kp) pred = FT<T>::flip(pred, bitp);
          const T p2 = REG ? regress<T, NDIM, OpV<T>>(cT, i, j, l) : wk.template combine<OpV<T>>();
          if (!FT<T>::same(pred, p2)) {
            pred = REG ? regress<T, NDIM, OpV<T>>(cT, i, j, l) : wk.template combine<OpV<T>>();
            ++r.dup;
          }
        }
        // lines 19-21: diff, quantization bin, range check (false for NaN / Inf)
        const T diff = FT<T>::sub(v, pred);
        const T t = FT<T>::mul(FT<T>::absv(diff), inv2);
        const bool inr = t < Rh;
        const int m = FT<T>::trunc_i(FT<T>::add(t, half));
        const int q = (diff < T(0)) ? -m : m;
        const T tq = FT<T>::fromi(2 * q);
        // line 25: dcmp <- dec_dup(q, pred')
        T xd = FT<T>::add(pred, FT<T>::mul(tq, eb));
        if (ABFT) {
          if (k == kr) xd = FT<T>::flip(xd, bitr);
          const T x2 = FT<T>::add_v(pred, FT<T>::mul_v(tq, eb));
          if (inr && !FT<T>::same(xd, x2)) {
            xd = FT<T>::add_v(pred, FT<T>::mul_v(tq, eb));
            ++r.dup;
          }
        }
        // lines 26-28: the reconstructed value must respect the bound, else unpredictable
        const bool ok = inr && (FT<T>::absv(FT<T>::sub(v, xd)) <= eb);
        const uint32_t code = ok ? (uint32_t)(q + (int)g.R) : 0u;
        const T xr = ok ? xd : v;
        codes[ci] = (uint16_t)code;
        if (!ok) {
          ustage[ci] = v;
          ++r.nun;
        }
        if (ABFT) {
          r.sq += code;  // line 24
          r.isq += (unsigned long long)(k + 1) * code;
          add_sum<T>(xr, r.sdc);  // line 29
        }
        if (code == run_code) {
          ++run_len;
        } else {
          if (run_len) h.add(run_code, run_len);
          run_code = code;
          run_len = 1;
        }
        if (!REG) wk.commit(j, l, xr);
      }
    }
  }
  if (run_len) h.add(run_code, run_len);
  return r;
}

template <typename T, int NDIM, bool ABFT>
__device__ __forceinline__ PassRes run_block(const T* field, const Geo& g, const Box& x, uint64_t b, bool reg,
                                             const T* cT, Walker<T, NDIM>& wk, T eb, T inv2, T Rh, uint16_t* codes,
                                             T* ustage, const Hist& h, uint32_t kp, uint32_t bitp, uint32_t kr,
                                             uint32_t bitr, uint32_t kfix, T xfix) {
  if (reg)
    return run_pass<T, NDIM, true, ABFT>(field, g, x, b, cT, wk, eb, inv2, Rh, codes, ustage, h, kp, bitp, kr, bitr,
                                         kfix, xfix);
  return run_pass<T, NDIM, false, ABFT>(field, g, x, b, cT, wk, eb, inv2, Rh, codes, ustage, h, kp, bitp, kr, bitr,
                                        kfix, xfix);
}

}  // namespace

template <typename T, int NDIM, bool ABFT>
__global__ void __launch_bounds__(128) k_predict(const T* __restrict__ field, Geo g, Ws w,
                                                 const sdcsz_flip* __restrict__ flips, uint32_t nflips) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  State* st = w.st;
  if (*(volatile unsigned int*)&st->error) return;
  const uint32_t tid = threadIdx.x;
  for (uint32_t q = tid; q < kHistWindow; q += blockDim.x) hist_s[q] = 0;
  __syncthreads();

  Hist h;
  h.s = hist_s;
  h.g = w.hist;
  h.lo = g.R > kHistWindow / 2 ? g.R - kHistWindow / 2 : 0;
  h.hi = min(g.bins, h.lo + (uint32_t)kHistWindow);

  const double ebd = st->eb;
  const T eb = (T)ebd;
  T inv2;
  if (sizeof(T) == 4) inv2 = (T)__double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, ebd)));
  else inv2 = (T)__ddiv_rn(1.0, __dmul_rn(2.0, ebd));
  const T Rh = FT<T>::sub(FT<T>::fromi((int)g.R), T(0.5));
  const float ebf = FT<T>::tofloat(eb);
  const float kappa = NDIM == 3 ? 1.22f : (NDIM == 2 ? 0.80f : 0.5f);
  const float noise = __fmul_rn(kappa, ebf);

  Walker<T, NDIM> wk;
  wk.base = reinterpret_cast<T*>(smem) + tid;
  wk.stride = blockDim.x;
  wk.B2 = g.B[2];
  wk.sr = g.B[1] * g.B[2];
  uint16_t* codes = w.codes;
  T* ustage = static_cast<T*>(w.ustage);
  T* coefT = static_cast<T*>(w.coefT);

  unsigned long long c_unpred = 0, c_reg = 0, c_dup = 0, c_fix = 0, c_bad = 0;
  const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + tid; b - tid < g.nb; b += step) {
    if (b >= g.nb) continue;
    const Box x = block_box(g, b);
    // line 8: indicator[i] <- the predictor with the smaller estimated error
    const float4 c4 = w.coef[b];
    const bool finite = w.pflag[b] & 1;
    bool reg = false;
    if (finite) {
      if (g.predictor == 2) reg = true;
      else if (g.predictor == 0) {
        const float2 e2 = w.est[b];
        reg = e2.x < __fadd_rn(e2.y, __fmul_rn((float)x.P, noise));
      }
    }
    T cT[4] = {FT<T>::fromfloat(c4.x), FT<T>::fromfloat(c4.y), FT<T>::fromfloat(c4.z), FT<T>::fromfloat(c4.w)};
    uint32_t kp = 0xffffffffu, bitp = 0, kr = 0xffffffffu, bitr = 0;
    if (nflips) {
      uint64_t idx;
      uint32_t bit;
      // every coefficient record of this block (after selection, before use)
      uint32_t lo = 0, hi = nflips;
      while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (flips[mid].block < b) lo = mid + 1;
        else hi = mid;
      }
      for (uint32_t t = lo; t < nflips && flips[t].block == b; ++t)
        if (flips[t].site == SDCSZ_SITE_COEF && flips[t].index <= (uint64_t)NDIM)
          cT[flips[t].index] = FT<T>::flip(cT[flips[t].index], flips[t].bit);
      if (ABFT && find_flip(flips, nflips, SDCSZ_SITE_PRED, b, &idx, &bit)) { kp = (uint32_t)idx; bitp = bit; }
      if (ABFT && find_flip(flips, nflips, SDCSZ_SITE_RECON, b, &idx, &bit)) { kr = (uint32_t)idx; bitr = bit; }
    }
    PassRes r = run_block<T, NDIM, ABFT>(field, g, x, b, reg, cT, wk, eb, inv2, Rh, codes, ustage, h, kp, bitp, kr,
                                         bitr, 0xffffffffu, T(0));
    uint8_t flag = reg ? 1 : 0;
    if (ABFT) {
      const unsigned long long s0 = w.sum_in[b], i0 = w.isum_in[b];
      if (r.sw != s0 || r.isw != i0) {
        // Alg. 1 line 11: locate the corrupted input word and repair it
        long long delta = 0;
        const long long m = locate_word(s0, i0, r.sw, r.isw, (unsigned long long)x.P * FT<T>::W, 0, &delta);
        bool fixed = false;
        if (m >= 0) {
          const uint32_t kf = (uint32_t)(m / FT<T>::W), wi = (uint32_t)(m % FT<T>::W);
          const uint32_t lf = kf % x.e[2], tq = kf / x.e[2];
          const uint32_t jf = tq % x.e[1], i_f = tq / x.e[1];
          const T cur = field[row_base(g, x, i_f, jf) + lf];
          uint32_t wd[2] = {FT<T>::lo(cur), FT<T>::hi(cur)};
          const long long nw = (long long)wd[wi] - delta;
          if (nw >= 0 && nw <= 0xffffffffll) {
            wd[wi] = (uint32_t)nw;
            const T xf = FT<T>::from_words(wd[0], wd[1]);
            // withdraw this block's first-pass codes from the histogram, then run it again
            uint64_t ci = code_index(b, g.P, 0);
            for (uint32_t kk = 0; kk < x.P; ++kk, ci += 32) h.sub1(codes[ci]);
            r = run_block<T, NDIM, ABFT>(field, g, x, b, reg, cT, wk, eb, inv2, Rh, codes, ustage, h, kp, bitp, kr,
                                         bitr, kf, xf);
            fixed = true;
            ++c_fix;
          }
        }
        if (!fixed) {
          ++c_bad;
          flag |= 2;
        }
      }
      w.sum_q[b] = r.sq;
      w.isum_q[b] = r.isq;
      w.sum_dc[b] = r.sdc;
    }
    w.flags[b] = flag;
    if (reg)
      for (int a = 0; a <= NDIM; ++a) coefT[4 * b + a] = cT[a];
    c_unpred += r.nun;
    c_reg += reg ? 1 : 0;
    c_dup += r.dup;
  }

  c_unpred = warp_sum(c_unpred);
  c_reg = warp_sum(c_reg);
  c_dup = warp_sum(c_dup);
  c_fix = warp_sum(c_fix);
  c_bad = warp_sum(c_bad);
  if ((tid & 31) == 0) {
    if (c_unpred) atomicAdd(&st->n_unpred, c_unpred);
    if (c_reg) atomicAdd(&st->n_reg, c_reg);
    if (c_dup) atomicAdd(&st->dup_fixed, c_dup);
    if (c_fix) atomicAdd(&st->input_corrected, c_fix);
    if (c_bad) atomicAdd(&st->uncorrectable, c_bad);
  }
  __syncthreads();
  for (uint32_t q = tid; q < h.hi - h.lo; q += blockDim.x)
    if (hist_s[q]) atomicAdd(&w.hist[h.lo + q], (unsigned long long)hist_s[q]);
}

template <typename T, int NDIM, bool ABFT>
static void run_predict(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L) {
  const uint32_t per = walker_slots(g.ndim, g.B) * sizeof(T);
  uint32_t threads = 128;
  while (threads > 32 && (size_t)per * threads > 160 * 1024) threads >>= 1;
  const size_t smem = (size_t)per * threads;
  auto kern = k_predict<T, NDIM, ABFT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (int)threads, smem);
  if (occ < 1) occ = 1;
  const uint64_t need = (g.nb + threads - 1) / threads;
  const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)occ * L.sms));
  kern<<<(unsigned)grid, threads, smem, L.stream>>>(static_cast<const T*>(field), g, w, flips, nflips);
}

void launch_predict(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                    const Launch& L) {
#define SDCSZ_P(T, N)                                                          \
  if (g.abft) run_predict<T, N, true>(field, g, w, flips, nflips, L);          \
  else run_predict<T, N, false>(field, g, w, flips, nflips, L);
  if (g.dtype == 0) {
    if (g.ndim == 3) { SDCSZ_P(float, 3) }
    else if (g.ndim == 2) { SDCSZ_P(float, 2) }
    else { SDCSZ_P(float, 1) }
  } else {
    if (g.ndim == 3) { SDCSZ_P(double, 3) }
    else if (g.ndim == 2) { SDCSZ_P(double, 2) }
    else { SDCSZ_P(double, 1) }
  }
#undef SDCSZ_P
}

// Soft-error simulation: flip bits of the caller's input after K1 took its checksums.
template <typename T>
__global__ void k_flip_input(T* field, Geo g, const sdcsz_flip* flips, uint32_t n) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (flips[t].site != SDCSZ_SITE_INPUT) continue;
    const uint64_t word = flips[t].index, pt = word / FT<T>::W;
    if (pt >= g.N) continue;
    uint32_t* wp = reinterpret_cast<uint32_t*>(field + pt) + (word % FT<T>::W);
    atomicXor(wp, 1u << (flips[t].bit & 31));
  }
}

void launch_flip_input(void* field, const Geo& g, const sdcsz_flip* flips, uint32_t nflips, const Ws& w,
                       const Launch& L) {
  (void)w;
  const unsigned grid = (nflips + 255) / 256;
  if (!grid) return;
  if (g.dtype == 0) k_flip_input<float><<<grid, 256, 0, L.stream>>>(static_cast<float*>(field), g, flips, nflips);
  else k_flip_input<double><<<grid, 256, 0, L.stream>>>(static_cast<double*>(field), g, flips, nflips);
}

// Soft-error simulation: flip bits of stored codes after their checksums were taken.
__global__ void k_flip_codes(Geo g, Ws w, const sdcsz_flip* flips, uint32_t n) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (flips[t].site != SDCSZ_SITE_CODE || flips[t].block >= g.nb) continue;
    const Box x = block_box(g, flips[t].block);
    if (flips[t].index >= x.P) continue;
    uint16_t* c = w.codes + code_index(flips[t].block, g.P, (uint32_t)flips[t].index);
    const uintptr_t a = reinterpret_cast<uintptr_t>(c);
    const uint32_t shift = (a & 2) ? 16u : 0u;
    atomicXor(reinterpret_cast<unsigned int*>(a & ~uintptr_t(3)), (1u << (flips[t].bit & 15)) << shift);
  }
}

void launch_flip_codes(const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips, const Launch& L) {
  const unsigned grid = (nflips + 255) / 256;
  if (!grid) return;
  k_flip_codes<<<grid, 256, 0, L.stream>>>(g, w, flips, nflips);
}

}  // namespace sdcsz
