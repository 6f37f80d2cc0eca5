// Internal definitions shared by the sdcsz CUDA kernels and the host entry points.
//
// Execution model (one GB300, sm_103a): every kernel maps one independent block (Sec. 5.1 of
// the paper) to one thread, and a warp to 32 consecutive blocks in row-major block order.
// Within a block the Lorenzo predictor depends on already reconstructed neighbours, so each
// thread walks its block point by point in the sequential order of the definition; the
// warp's lanes run 32 such walks side by side. Neighbour values live in a per-thread slice of
// shared memory laid out slot-major ([slot][thread]) so a warp's accesses are conflict free.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sdcsz.h"

namespace sdcsz {

constexpr int kMaxLen = 24;           // longest Huffman code in bits
constexpr int kGroup = 256;           // blocks per random-access group of the stream
constexpr int kHeaderBytes = 128;
constexpr int kLutBits = 12;          // first-level decode table covers codes of <= 12 bits
constexpr int kHistWindow = 2048;     // bins privatised in shared memory around the centre
constexpr uint32_t kSpinLimit = 1u << 20;  // bounded waits: iterations before giving up

// error flags accumulated in State::error
enum : uint32_t { ERR_EB = 1u, ERR_CAPACITY = 2u, ERR_TIMEOUT = 4u, ERR_FORMAT = 8u, ERR_FIELD = 16u };

// Geometry and parameters, padded to 3D with leading unit dimensions; passed by value.
struct Geo {
  int ndim, dtype;
  uint64_t d[3];
  uint32_t B[3];
  uint64_t nbd[3];
  uint64_t nb, N;
  uint32_t P;  // points in a full block
  uint32_t bins, R;
  int abft, predictor, eb_mode;
  int enc;       // 1: compact encoding (coefficients and unpredictable values in the payload)
  int lossless;  // 1: the lossless stage codes the stream after its block tables
  double e;
  // block-index decomposition without a division (fields of fewer than 2^32 blocks):
  // floor(n / nbd[a]) = mulhi64(rcp[a], n) for every 32-bit n, rcp[a] = ceil(2^64 / nbd[a])
  // (Lemire, Kaser, Kurz, "Faster remainder by direct computation", 2019); 0 for nbd[a] = 1
  uint64_t rcp[3];
};

// The reciprocals of the block counts along each axis (host side, after nbd is set).
inline void geo_rcp(Geo* g) {
  for (int a = 0; a < 3; ++a) g->rcp[a] = (g->nbd[a] > 1 && g->nbd[a] <= 0xffffffffull) ? ~0ull / g->nbd[a] + 1 : 0ull;
}

// floor(n / d) for the 32-bit n of a field of fewer than 2^32 blocks (rcp from geo_rcp)
__device__ __forceinline__ uint32_t div_rcp(uint32_t n, uint64_t rcp) {
  return rcp ? (uint32_t)__umul64hi(rcp, (unsigned long long)n) : n;
}

// Block b's coordinates in the block grid (row-major, the fastest axis last).
__device__ __forceinline__ void block_coords(const Geo& g, uint64_t b, uint64_t& c0, uint64_t& c1, uint64_t& c2) {
  if (g.nb <= 0xffffffffull) {
    const uint32_t bb = (uint32_t)b, n2 = (uint32_t)g.nbd[2], n1 = (uint32_t)g.nbd[1];
    const uint32_t t = div_rcp(bb, g.rcp[2]);
    const uint32_t q = div_rcp(t, g.rcp[1]);
    c2 = bb - t * n2;
    c1 = t - q * n1;
    c0 = q;
  } else {
    c2 = b % g.nbd[2];
    const uint64_t t = b / g.nbd[2];
    c1 = t % g.nbd[1];
    c0 = t / g.nbd[1];
  }
}

// Byte offsets of the stream sections (16-byte aligned).
struct Layout {
  uint64_t table, groups, sizes, ucounts, bitmap, sumdc, coef, unpred, payload;
};

// Device-side state of one call; lives at the start of the workspace.
struct State {
  unsigned long long min_key, max_key;
  unsigned int k1_done;
  unsigned int error;
  double eb;  // absolute bound, the dtype value widened to double
  unsigned long long n_reg, n_unpred;
  unsigned long long input_corrected, codes_corrected, dup_fixed, uncorrectable, reexec_corrected, bound_viol;
  unsigned long long max_err_bits;  // double bits of max |x - x'| (non-negative: ordered as u64)
  unsigned int ticket, n_live;
  unsigned long long payload_bytes, total_bytes;
  unsigned long long n_unpred_enc;  // unpredictable points of the codes as encoded (after repairs)
  double cstep[4], cinv[4];         // compact encoding: coefficient steps (set with the bound)
  unsigned long long raw_total;     // lossless stage: size of the stream before the stage
  Layout L;
  unsigned long long queue[4];  // work-queue counters of the persistent kernels of one call
};

// Work queue of a persistent kernel: the CTA takes the next item index (one atomic per CTA).
// Items go to the CTAs that are running, so a grid that cannot be resident at once (other
// kernels hold some of the SMs' slots) still finishes when its running CTAs have drained it.
__device__ __forceinline__ uint64_t cta_pull(unsigned long long* q) {
  __shared__ unsigned long long s_item_q;
  __syncthreads();
  if (threadIdx.x == 0) s_item_q = atomicAdd(q, 1ull);
  __syncthreads();
  return s_item_q;
}

// Totals the per-block encoder sums for the stream assembly (64-bit atomics per warp): one word
// per group of kGroup blocks, regression blocks << 46 | unpredictables << 25 | payload bytes
// (at most 256, 2^20 and 256 * 65535 < 2^25: no field carries into the next), then two words
// per super-group of kSuper groups: payload bytes, and unpredictables << 17 | regression
// blocks (at most 2^28 and 2^16).
constexpr uint64_t kSuper = 256;
__host__ __device__ inline uint64_t group_total_words(uint64_t ngroups) {
  return ngroups + 2 * ((ngroups + kSuper - 1) / kSuper);
}

// Pointers into a compress workspace.
struct Ws {
  State* st;
  unsigned long long *sum_in, *isum_in, *sum_q, *isum_q, *sum_dc;
  float4* coef;        // fp32 regression coefficients per block
  float2* est;         // (E_reg, E_lor) per block
  uint8_t* pflag;      // bit0: coefficients finite
  uint8_t* flags;      // bit0: regression block, bit1: input uncorrectable
  void* coefT;         // dtype coefficients used by regression blocks (4 per block)
  unsigned long long* hist;
  uint32_t* codebook;  // code << 5 | length per symbol
  unsigned long long* gt;  // group and super-group totals (group_total_words)
  unsigned long long* sort_keys;  // codebook construction scratch
  unsigned long long* node_w;
  uint32_t* node_parent;
  uint16_t* codes;     // quantization codes in warp-interleaved pairs (see pair_index)
  void* ustage;        // unpredictable values, same interleaving as codes
  uint32_t* etmp;      // per-block payload slots of the encoder (encode_slot_words each)
  // lossless stage (compression): the stream before the stage and the coder's scratch
  uint8_t* raw;                    // the stream before the stage (raw_cap bytes)
  unsigned long long raw_cap;
  uint16_t* llw;                   // per chunk: kLLChunk words, filled from the end
  uint32_t* llst;                  // per chunk: 32 final states
  uint32_t* llsz;                  // per chunk: coded bytes (padded to 4); then the first word used
  uint32_t* lltop;
  unsigned long long* lloff;       // per chunk: offset in the output
  unsigned long long* llhist;      // byte histogram (256)
  uint32_t* llcum;                 // cumulative frequencies (257)
};

// Lossless stage: order-0 rANS over the bytes after the block tables, in independent chunks
// of kLLChunk bytes, 32 interleaved states each (byte i of a chunk belongs to state i mod 32).
constexpr uint32_t kLLChunk = 16384, kLLScale = 12, kLLM = 1u << kLLScale, kLLTable = 512;

__host__ __device__ inline uint64_t align16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

__host__ __device__ inline Layout make_layout(const Geo& g, uint64_t n_live, uint64_t n_reg, uint64_t n_unpred) {
  const uint64_t s = g.dtype ? 8 : 4;
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  Layout L;
  L.table = kHeaderBytes;
  L.groups = align16(L.table + 4 * (kMaxLen + 1) + 2 * n_live);
  L.sizes = align16(L.groups + 24 * ngroups);
  L.ucounts = align16(L.sizes + 2 * g.nb);
  L.bitmap = align16(L.ucounts + 2 * g.nb);
  L.sumdc = align16(L.bitmap + 4 * ((g.nb + 31) / 32));
  L.coef = align16(L.sumdc + (g.abft ? 8 * g.nb : 0));
  L.unpred = align16(L.coef + (g.enc ? 0 : s * (uint64_t)(g.ndim + 1) * n_reg));
  L.payload = align16(L.unpred + (g.enc ? 0 : s * n_unpred));
  return L;
}

__host__ __device__ inline uint64_t code_index(uint64_t b, uint32_t P, uint32_t k) {
  return ((b >> 5) * (uint64_t)P + k) * 32 + (b & 31);
}

// Quantization codes are staged in pairs: the 32-bit word pair_index(b, P, k) holds the codes
// of points k & ~1 (low half) and k | 1 (high half) of block b, warp-interleaved so that a
// warp's 32 lanes (32 consecutive blocks) move 128 contiguous bytes per instruction.
__host__ __device__ inline uint32_t pairs_of(uint32_t P) { return (P + 1) / 2; }
__host__ __device__ inline uint64_t pair_index(uint64_t b, uint32_t P, uint32_t k) {
  return ((b >> 5) * (uint64_t)pairs_of(P) + (k >> 1)) * 32 + (b & 31);
}
__host__ __device__ inline uint64_t code_pos(uint64_t b, uint32_t P, uint32_t k) {
  return 2 * pair_index(b, P, k) + (k & 1);
}

// Block b's origin and extents (edge blocks are cut to the field).
struct Box {
  uint64_t org[3];
  uint32_t e[3];
  uint32_t P;
};

__device__ __forceinline__ Box block_box(const Geo& g, uint64_t b) {
  Box x;
  uint64_t c0, c1, c2;
  block_coords(g, b, c0, c1, c2);
  x.org[0] = c0 * g.B[0];
  x.org[1] = c1 * g.B[1];
  x.org[2] = c2 * g.B[2];
  x.e[0] = (uint32_t)min((uint64_t)g.B[0], g.d[0] - x.org[0]);
  x.e[1] = (uint32_t)min((uint64_t)g.B[1], g.d[1] - x.org[1]);
  x.e[2] = (uint32_t)min((uint64_t)g.B[2], g.d[2] - x.org[2]);
  x.P = x.e[0] * x.e[1] * x.e[2];
  return x;
}

// Edge blocks (cut by the field boundary) enumerated compactly, so a warp gets 32 of them:
// the slab c0 = last (when dims[0] is not a multiple), then c1 = last, then c2 = last.
__host__ __device__ inline uint64_t edge_count(const Geo& g) {
  const uint64_t p0 = g.d[0] % g.B[0] != 0, p1 = g.d[1] % g.B[1] != 0, p2 = g.d[2] % g.B[2] != 0;
  const uint64_t F0 = g.nbd[0] - p0, F1 = g.nbd[1] - p1;
  return p0 * g.nbd[1] * g.nbd[2] + F0 * p1 * g.nbd[2] + F0 * F1 * p2;
}

__device__ __forceinline__ uint64_t edge_block(const Geo& g, uint64_t e) {
  const uint64_t p0 = g.d[0] % g.B[0] != 0, p1 = g.d[1] % g.B[1] != 0;
  const uint64_t F0 = g.nbd[0] - p0, F1 = g.nbd[1] - p1, F2 = g.nbd[2] - (g.d[2] % g.B[2] != 0);
  const uint64_t A = p0 * g.nbd[1] * g.nbd[2], Bn = F0 * p1 * g.nbd[2];
  uint64_t c0, c1, c2;
  if (e < A) {
    const uint64_t r = e % (g.nbd[1] * g.nbd[2]);
    c0 = F0 + e / (g.nbd[1] * g.nbd[2]);
    c1 = r / g.nbd[2];
    c2 = r % g.nbd[2];
  } else if (e < A + Bn) {
    const uint64_t r = e - A;
    c0 = r / g.nbd[2];
    c1 = F1;
    c2 = r % g.nbd[2];
  } else {
    const uint64_t r = e - A - Bn;
    c0 = r / F1;
    c1 = r % F1;
    c2 = F2;
  }
  return (c0 * g.nbd[1] + c1) * g.nbd[2] + c2;
}

// Rows of the predictor-selection sample (whole rows along the fastest axis): one diagonal
// row per plane in 3D, every fourth row from row 1 in 2D, the whole block in 1D.
__host__ __device__ inline bool sample_row(int ndim, uint32_t i, uint32_t j, uint32_t e1) {
  if (ndim == 3) return j == i % e1;
  if (ndim == 2) return (j & 3u) == 1u;
  return true;
}

__host__ __device__ inline uint32_t sample_points(int ndim, const uint32_t e[3]) {
  if (ndim == 3) return e[0] * e[2];
  if (ndim == 2) return ((e[1] + 2) / 4) * e[2];
  return e[2];
}

__device__ __forceinline__ uint64_t row_base(const Geo& g, const Box& x, uint32_t i, uint32_t j) {
  return ((x.org[0] + i) * g.d[1] + (x.org[1] + j)) * g.d[2] + x.org[2];
}

// ---------------------------------------------------------------- typed arithmetic
// Every value-producing operation is an explicitly rounded IEEE operation (no contraction).
// The *_v variants are volatile inline PTX: the duplicated evaluations of Algorithm 1 (f_dup
// and dec_dup) cannot be merged with the primary ones by the compiler.
template <typename T> struct FT;

template <> struct FT<float> {
  static constexpr int W = 1;
  __device__ static __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ static __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  __device__ static __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ static __forceinline__ float add_v(float a, float b) {
    float r; asm volatile("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b)); return r;
  }
  __device__ static __forceinline__ float sub_v(float a, float b) {
    float r; asm volatile("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b)); return r;
  }
  __device__ static __forceinline__ float mul_v(float a, float b) {
    float r; asm volatile("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b)); return r;
  }
  __device__ static __forceinline__ float fromi(int v) { return __int2float_rn(v); }
  __device__ static __forceinline__ int trunc_i(float v) { return __float2int_rz(v); }
  __device__ static __forceinline__ float absv(float v) { return fabsf(v); }
  __device__ static __forceinline__ bool same(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
  // zero iff a and b have the same bits
  __device__ static __forceinline__ uint32_t diffbits(float a, float b) { return __float_as_uint(a) ^ __float_as_uint(b); }
  __device__ static __forceinline__ float flip(float v, uint32_t bit) { return __uint_as_float(__float_as_uint(v) ^ (1u << (bit & 31))); }
  __device__ static __forceinline__ uint32_t lo(float v) { return __float_as_uint(v); }
  __device__ static __forceinline__ uint32_t hi(float) { return 0u; }
  __device__ static __forceinline__ float from_words(uint32_t lo, uint32_t) { return __uint_as_float(lo); }
  __device__ static __forceinline__ bool finite(float v) { return isfinite(v); }
  __device__ static __forceinline__ float tofloat(float v) { return v; }
  __device__ static __forceinline__ float fromfloat(float v) { return v; }
  // monotone unsigned key: a < b  <=>  key(a) < key(b) (for non-NaN)
  __device__ static __forceinline__ unsigned long long key(float v) {
    uint32_t u = __float_as_uint(v);
    return (unsigned long long)((u & 0x80000000u) ? ~u : (u | 0x80000000u));
  }
  __device__ static __forceinline__ float unkey(unsigned long long k) {
    uint32_t u = (uint32_t)k;
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
  }
  __device__ static __forceinline__ bool is_normal_pos(float v) { return v >= 1.17549435e-38f && v <= 3.40282347e38f; }
};

template <> struct FT<double> {
  static constexpr int W = 2;
  __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  __device__ static __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ static __forceinline__ double add_v(double a, double b) {
    double r; asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b)); return r;
  }
  __device__ static __forceinline__ double sub_v(double a, double b) {
    double r; asm volatile("sub.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b)); return r;
  }
  __device__ static __forceinline__ double mul_v(double a, double b) {
    double r; asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b)); return r;
  }
  __device__ static __forceinline__ double fromi(int v) { return __int2double_rn(v); }
  __device__ static __forceinline__ int trunc_i(double v) { return __double2int_rz(v); }
  __device__ static __forceinline__ double absv(double v) { return fabs(v); }
  __device__ static __forceinline__ bool same(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }
  __device__ static __forceinline__ uint32_t diffbits(double a, double b) {
    const unsigned long long d = (unsigned long long)(__double_as_longlong(a) ^ __double_as_longlong(b));
    return (uint32_t)d | (uint32_t)(d >> 32);
  }
  __device__ static __forceinline__ double flip(double v, uint32_t bit) {
    return __longlong_as_double(__double_as_longlong(v) ^ (1ll << (bit & 63)));
  }
  __device__ static __forceinline__ uint32_t lo(double v) { return (uint32_t)(unsigned long long)__double_as_longlong(v); }
  __device__ static __forceinline__ uint32_t hi(double v) { return (uint32_t)((unsigned long long)__double_as_longlong(v) >> 32); }
  __device__ static __forceinline__ double from_words(uint32_t lo, uint32_t hi) {
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
  }
  __device__ static __forceinline__ bool finite(double v) { return isfinite(v); }
  __device__ static __forceinline__ float tofloat(double v) { return __double2float_rn(v); }
  __device__ static __forceinline__ double fromfloat(float v) { return (double)v; }
  __device__ static __forceinline__ unsigned long long key(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
  }
  __device__ static __forceinline__ double unkey(unsigned long long k) {
    return __longlong_as_double((long long)((k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k));
  }
  __device__ static __forceinline__ bool is_normal_pos(double v) { return v >= 2.2250738585072014e-308 && v <= 1.7976931348623157e308; }
};

// ---------------------------------------------------------------- compact encoding
// Bit fields of the dtype (mantissa bits, exponent bits, bias) and the value as an integer.
template <typename T> struct Bitsof;
template <> struct Bitsof<float> {
  typedef uint32_t U;
  static constexpr int M = 23, E = 8, BIAS = 127;
  __device__ static __forceinline__ U raw(float v) { return __float_as_uint(v); }
  __device__ static __forceinline__ float val(U u) { return __uint_as_float(u); }
};
template <> struct Bitsof<double> {
  typedef unsigned long long U;
  static constexpr int M = 52, E = 11, BIAS = 1023;
  __device__ static __forceinline__ U raw(double v) { return (U)__double_as_longlong(v); }
  __device__ static __forceinline__ double val(U u) { return __longlong_as_double((long long)u); }
};

// floor(log2(eb)) of the dtype bound eb (normal); kNoTrunc keeps every mantissa bit.
constexpr int kNoTrunc = -100000;
template <typename T>
__device__ __forceinline__ int bound_exponent(T eb) {
  return (int)((Bitsof<T>::raw(eb) >> Bitsof<T>::M) & ((1u << Bitsof<T>::E) - 1)) - Bitsof<T>::BIAS;
}

// Mantissa bits an unpredictable value keeps so that dropping the rest errs by less than
// 2^texp <= eb: with v in [2^ex, 2^(ex+1)) that is ex - texp bits, clamped to [0, M]; zeros,
// subnormals, infinities and NaNs keep all of them.
template <typename T>
__device__ __forceinline__ int kept_bits(T v, int texp) {
  const int Ex = (int)((Bitsof<T>::raw(v) >> Bitsof<T>::M) & ((1u << Bitsof<T>::E) - 1));
  if (Ex == 0 || Ex == (1 << Bitsof<T>::E) - 1) return Bitsof<T>::M;
  return min(max(Ex - Bitsof<T>::BIAS - texp, 0), Bitsof<T>::M);
}

// The value an unpredictable point decompresses to (v itself when texp is kNoTrunc).
template <typename T>
__device__ __forceinline__ T truncated(T v, int texp) {
  const int drop = Bitsof<T>::M - kept_bits<T>(v, texp);
  typedef typename Bitsof<T>::U U;
  return Bitsof<T>::val(Bitsof<T>::raw(v) & ~((((U)1) << drop) - (U)1));
}

// Steps of the coefficient integers: slope a (of ndim) eb / (16 B_a), intercept eb / 16, for
// the absolute bound E (the dtype value widened); inverse steps for the rounding.
struct CoefSteps {
  double step[4], inv[4];
};
__host__ __device__ inline CoefSteps coef_steps(const Geo& g, double E) {
  CoefSteps q;
  const int off = 3 - g.ndim;
  for (int a = 0; a < 4; ++a) q.step[a] = q.inv[a] = 0.0;
  for (int a = 0; a < g.ndim; ++a) {
    const double d = 16.0 * (double)g.B[off + a];
    q.step[a] = E / d;
    q.inv[a] = d / E;
  }
  q.step[g.ndim] = E / 16.0;
  q.inv[g.ndim] = 16.0 / E;
  return q;
}

// Nearest multiple of the step, halves away from zero; false unless below 2^30 steps.
__device__ __forceinline__ bool coef_to_int(float c, double inv, int* k) {
  const double t = __dmul_rn((double)c, inv);
  if (!(fabs(t) < 1073741824.0)) return false;
  const double m = floor(__dadd_rn(fabs(t), 0.5));
  *k = (int)(t < 0.0 ? -m : m);
  return true;
}

template <typename T>
__device__ __forceinline__ T coef_from_int(int k, double step) {
  const double v = __dmul_rn((double)k, step);
  if (sizeof(T) == 4) return (T)__double2float_rn(v);
  return (T)v;
}

// Checksum words of one value at point k: sum += words, isum += (word index + 1) * word
// (Sec. 3.2 and 5.4; float64 = two 32-bit words, low word first).
template <typename T>
__device__ __forceinline__ void add_words(T v, uint32_t k, unsigned long long& sum, unsigned long long& isum) {
  const uint32_t w0 = FT<T>::lo(v);
  if (FT<T>::W == 1) {
    sum += w0;
    isum += (unsigned long long)(k + 1) * w0;
  } else {
    const uint32_t w1 = FT<T>::hi(v);
    sum += (unsigned long long)w0 + w1;
    isum += (unsigned long long)(2 * k + 1) * w0 + (unsigned long long)(2 * k + 2) * w1;
  }
}

template <typename T>
__device__ __forceinline__ void add_sum(T v, unsigned long long& sum) {
  if (FT<T>::W == 1) sum += FT<T>::lo(v);
  else sum += (unsigned long long)FT<T>::lo(v) + FT<T>::hi(v);
}

// Sec. 3.2: given the stored (sum0, isum0) and the recomputed (sum1, isum1), locate a single
// changed word: its 1-based index is (isum1 - isum0) / (sum1 - sum0). Returns the 0-based
// word index and the repaired word, or -1 when no single-word explanation exists.
__device__ __forceinline__ long long locate_word(unsigned long long sum0, unsigned long long isum0,
                                                 unsigned long long sum1, unsigned long long isum1,
                                                 unsigned long long nwords, uint32_t cur_word_unknown,
                                                 long long* delta_out) {
  long long ds = (long long)(sum1 - sum0);
  long long dis = (long long)(isum1 - isum0);
  (void)cur_word_unknown;
  if (ds == 0) return -1;
  if (dis % ds != 0) return -1;
  long long pos = dis / ds;
  if (pos < 1 || (unsigned long long)pos > nwords) return -1;
  *delta_out = ds;
  return pos - 1;
}

// ---------------------------------------------------------------- predictors
// Lorenzo predictor over reconstructed neighbours with zero outside the block, walked in the
// block's sequential (row-major) order. The previous plane (3D) / row (2D) sits in this
// thread's shared-memory slots; the previous point's neighbours stay in registers.
//   3D: pred = ((((((a + b) - ab) - ac) - bc) + abc) + c) with a = d[i-1,j,l],
//       b = d[i,j-1,l], c = d[i,j,l-1], ab = d[i-1,j-1,l], ac = d[i-1,j,l-1],
//       bc = d[i,j-1,l-1], abc = d[i-1,j-1,l-1].
//   2D: pred = (d[j-1,l] - d[j-1,l-1]) + d[j,l-1].   1D: pred = d[l-1].
// The previous point of the row (c) comes last: it is the only operand that depends on the
// point just reconstructed, so the serial chain per point is a single addition before the
// quantizer.
template <typename V, int NDIM>
struct Walker {
  V* base;        // this thread's slot 0
  uint32_t stride;
  uint32_t B2;    // slots per plane row
  uint32_t sr;    // first slot of the saved row (3D)
  V a, b, ab;     // neighbours loaded for the current point
  V ap, bp, abp, cp;  // the same at l-1, and the previous reconstructed value

  __device__ __forceinline__ V& slot(uint32_t s) { return base[(size_t)s * stride]; }
  __device__ __forceinline__ void row_start() { ap = bp = abp = cp = V(0); }

  template <class Op>
  __device__ __forceinline__ V combine() const {
    if (NDIM == 3) {
      V s = Op::add(a, b);
      s = Op::sub(s, ab);
      s = Op::sub(s, ap);
      s = Op::sub(s, bp);
      s = Op::add(s, abp);
      return Op::add(s, cp);
    } else if (NDIM == 2) {
      V s = Op::sub(a, ap);
      return Op::add(s, cp);
    } else {
      return cp;
    }
  }
  __device__ __forceinline__ void load(uint32_t i, uint32_t j, uint32_t l) {
    if (NDIM == 3) {
      a = (i > 0) ? slot(j * B2 + l) : V(0);
      b = (j > 0) ? slot((j - 1) * B2 + l) : V(0);
      ab = (i > 0 && j > 0) ? slot(sr + l) : V(0);
    } else if (NDIM == 2) {
      a = (j > 0) ? slot(l) : V(0);
    }
  }
  __device__ __forceinline__ void commit(uint32_t j, uint32_t l, V x) {
    if (NDIM == 3) {
      slot(sr + l) = a;
      slot(j * B2 + l) = x;
      ap = a;
      bp = b;
      abp = ab;
    } else if (NDIM == 2) {
      slot(l) = x;
      ap = a;
    }
    cp = x;
  }
};

template <typename T> struct OpRN {
  __device__ static __forceinline__ T add(T a, T b) { return FT<T>::add(a, b); }
  __device__ static __forceinline__ T sub(T a, T b) { return FT<T>::sub(a, b); }
  __device__ static __forceinline__ T mul(T a, T b) { return FT<T>::mul(a, b); }
};
template <typename T> struct OpV {
  __device__ static __forceinline__ T add(T a, T b) { return FT<T>::add_v(a, b); }
  __device__ static __forceinline__ T sub(T a, T b) { return FT<T>::sub_v(a, b); }
  __device__ static __forceinline__ T mul(T a, T b) { return FT<T>::mul_v(a, b); }
};

// Per-thread shared-memory slots the Lorenzo walk needs for a block shape.
__host__ __device__ inline uint32_t walker_slots(int ndim, const uint32_t B[3]) {
  if (ndim == 3) return B[1] * B[2] + B[2];
  if (ndim == 2) return B[2];
  return 0;
}

// Regression predictor ((b0*c0 + b1*c1) + b2*c2) + b_n over the block's own coordinates.
template <typename V, int NDIM, class Op>
__device__ __forceinline__ V regress(const V* c, uint32_t i, uint32_t j, uint32_t l) {
  if (NDIM == 3) {
    V acc = Op::mul(c[0], (V)i);
    acc = Op::add(acc, Op::mul(c[1], (V)j));
    acc = Op::add(acc, Op::mul(c[2], (V)l));
    return Op::add(acc, c[3]);
  } else if (NDIM == 2) {
    V acc = Op::mul(c[0], (V)j);
    acc = Op::add(acc, Op::mul(c[1], (V)l));
    return Op::add(acc, c[2]);
  } else {
    V acc = Op::mul(c[0], (V)l);
    return Op::add(acc, c[1]);
  }
}

// Look up the first soft-error record of `site` for block b in a list sorted by block.
__device__ __forceinline__ bool find_flip(const sdcsz_flip* f, uint32_t n, uint32_t site, uint64_t b,
                                          uint64_t* index, uint32_t* bit) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (f[mid].block < b) lo = mid + 1;
    else hi = mid;
  }
  for (uint32_t t = lo; t < n && f[t].block == b; ++t)
    if (f[t].site == site) {
      *index = f[t].index;
      *bit = f[t].bit;
      return true;
    }
  return false;
}

// Ask the memory system to bring the 128-byte line holding p into L2 ahead of its use (no
// register is written and nothing waits on it). Callers pass addresses inside their buffers.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- host-side launchers
struct Launch {
  cudaStream_t stream;
  int sms;
};

// Counts every kernel launch the library issues (read back by sdcsz_kernel_launches).
void note_launch();

// A library-owned stream for work that overlaps the caller's stream `main`: one per
// (device, caller stream), so concurrent callers on different streams never share one.
cudaStream_t side_stream(cudaStream_t main);

// Resident CTAs per SM of `kern` at (threads, smem), cached per device; also raises the
// kernel's dynamic shared-memory limit to `smem` once. Host-side launch setup only.
int occupancy(const void* kern, int threads, size_t smem);
void allow_smem(const void* kern, size_t smem);

// Fork/join: work launched on `side` runs concurrently with the caller's stream between the
// constructor and join(); join() makes the caller's stream wait for it. Events carry the
// dependencies, so this also works while the caller's stream is being captured into a graph.
struct Fork {
  cudaStream_t main = nullptr, side = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool on = false;
  explicit Fork(const Launch& L) : main(L.stream) {
    side = side_stream(main);
    if (!side || cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess) return;
    if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) return;
    cudaEventRecord(e0, main);
    cudaStreamWaitEvent(side, e0, 0);
    on = true;
  }
  Launch side_launch(const Launch& L) const {
    Launch s = L;
    if (on) s.stream = side;
    return s;
  }
  void join() {
    if (on) {
      cudaEventRecord(e1, side);
      cudaStreamWaitEvent(main, e1, 0);
      on = false;
    }
  }
  ~Fork() {
    join();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

void launch_prep(const void* field, const Geo& g, const Ws& w, const Launch& L);
// The absolute bound from the range keys in the State (the last kernel of launch_prep).
void launch_bound(const Geo& g, State* st, const Launch& L);
void launch_predict(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                    const Launch& L);
void launch_flip_input(void* field, const Geo& g, const sdcsz_flip* flips, uint32_t nflips, const Ws& w,
                       const Launch& L);
void launch_flip_codes(const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips, const Launch& L);
void launch_codebook(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L);
void launch_encode(const void* field, const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L);

// A slab of a field compressed as one shard of the field's stream (sharded compression over
// several GPUs). The slab is a field of its own to every kernel up to the encoder; the encoder
// places its blocks in the field's stream: block b of the slab is block boff + b of the field,
// and its payload, unpredictable values and coefficients follow those of the earlier shards
// (pre: their payload bytes, unpredictable values and regression blocks). tot: the field's
// payload bytes, unpredictable values, regression blocks and uncorrectable blocks. Only the
// shard with header = 1 writes the header and the code table. on = 0: a whole field.
struct Shard {
  int on, header;
  uint64_t boff;
  unsigned long long pre[3], tot[4];
};
// K4a of a shard into `out` at the field's layout (State::L, set by the codebook kernel from the
// field's geometry), then K4b with the shard's offsets.
void launch_encode_shard_blocks(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Shard& sh,
                                const Launch& L);
void launch_encode_shard_assemble(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Shard& sh,
                                  const Launch& L);

// ---------------------------------------------------------------- batches
// A batch compresses many fields with one launch per stage and kernel shape: every field is
// a Job in a device-side table, and the CTAs of a persistent launch pull work items (a field
// and a range of its blocks) from a queue counter in device memory. A field's items are
// numbered from 0 like the CTAs of a single-field launch, so the same per-item code runs in
// both cases and a field's output is the same alone and in a batch.
constexpr int kMaxBatch = 64;    // fields per batch
constexpr int kMaxQueues = 64;   // queue counters per batch (one per launch)

struct Job {
  Geo g;
  Ws w;
  const void* field;
  uint8_t* out;
  uint64_t cap;
  int vec2;        // the field's rows allow two-value vector loads
  int fast;        // the block shape has a compile-time fast path
  uint64_t gcount; // blocks of the generic path: edge blocks, or all blocks without a fast path
};

// One batched launch: the jobs it serves and the first item of each.
struct BatchArgs {
  const Job* jobs;
  unsigned long long* head;         // this launch's queue counter (zero before the launch)
  uint32_t n;
  uint32_t idx[kMaxBatch];          // job table indices
  uint64_t start[kMaxBatch + 1];    // item prefix sums; start[n] = items in the launch
};

__device__ __forceinline__ uint32_t find_job(const BatchArgs& a, uint64_t item) {
  uint32_t lo = 0, hi = a.n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a.start[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The CTA loop of a batched launch: pull an item, make its job current in shared memory
// (calling leave() for the previous job and enter() for the new one; both run on every
// thread), skip jobs whose call already failed, and run body(local item index). Every
// decision is taken once per CTA and broadcast, so the body's barriers stay uniform. A CTA
// may find the queue drained at its first pull (others started earlier and took every item):
// it then leaves without touching any job.
template <class Enter, class Body, class Leave>
__device__ __forceinline__ void batch_loop(const BatchArgs& a, Job& s_job, Enter&& enter, Body&& body,
                                           Leave&& leave) {
  __shared__ unsigned long long s_item;
  __shared__ int s_cur, s_skip;
  if (threadIdx.x == 0) s_cur = -1;
  const uint64_t total = a.start[a.n];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1ull);
    __syncthreads();
    const uint64_t item = s_item;
    const int cur = s_cur;
    if (item >= total) {  // queue drained (possibly before this CTA got any item)
      if (cur >= 0) leave();
      break;
    }
    const int j = (int)find_job(a, item);
    if (j != cur) {
      if (cur >= 0) leave();
      __syncthreads();
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&a.jobs[a.idx[j]]);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_job);
      for (uint32_t q = threadIdx.x; q < sizeof(Job) / 8; q += blockDim.x) dst[q] = src[q];
      __syncthreads();
      if (threadIdx.x == 0) s_cur = j;
      enter();
    }
    if (threadIdx.x == 0) s_skip = *(volatile unsigned int*)&s_job.w.st->error != 0;
    __syncthreads();
    if (!s_skip) body(item - a.start[j]);
  }
}

struct NoOp {
  __device__ __forceinline__ void operator()() const {}
};

// Batched launches (one per stage and kernel shape; see BatchArgs).
bool prep_has_fast(const Geo& g);
// Blocks per CTA group of the wavefront kernels for cube edge B (0: none). Prediction takes
// them for 12^3 and 16^3 (wave_predicts); 10^3 predicts faster one thread per block on smooth
// fields, where nearly every row is a central row (0.44 against 0.87 ms at 512^3).
__host__ __device__ constexpr uint32_t wave_group_blocks(uint32_t B) { return B == 16 ? 8 : (B == 10 || B == 12) ? 16 : 0; }
__host__ __device__ constexpr bool wave_predicts(uint32_t B) { return B == 12 || B == 16; }
// The two-pass decoder of those shapes keeps, per block: its code pairs and unpredictable values
// at the compression's interleaved places (a full block's stride), four coefficients, a flag
// byte and a re-execution list entry. wave_dws_part(g, i) is part i's size (i < 5).
inline uint64_t wave_dws_part(const Geo& g, int i) {
  const uint64_t P = g.P, nb32 = (g.nb + 31) / 32 * 32, es = g.dtype ? 8 : 4;
  const uint64_t n[5] = {nb32 * pairs_of((uint32_t)P) * 4, nb32 * P * es, g.nb * 4 * es, g.nb, g.nb * 8};
  return (n[i] + 255) & ~uint64_t(255);
}
inline uint64_t wave_decode_ws_bytes(const Geo& g) {  // 0 for shapes the two-pass decoder does not serve
  if (g.ndim != 3 || g.B[0] != g.B[1] || g.B[1] != g.B[2] || !wave_group_blocks(g.B[2]) || !g.nb) return 0;
  if (g.B[2] != 16 && g.dtype == 0) return 0;  // 10^3 and 12^3 float32 decode in one pass
  uint64_t t = 0;
  for (int i = 0; i < 5; ++i) t += wave_dws_part(g, i);
  return t;
}
inline uint64_t wave_groups(const Geo& g) {  // 0 unless g's blocks take the wavefront kernel
  if (g.ndim != 3 || g.B[0] != g.B[1] || g.B[1] != g.B[2] || !wave_predicts(g.B[2])) return 0;
  const uint64_t G = wave_group_blocks(g.B[2]);
  return G ? (g.nb + G - 1) / G + (edge_count(g) + G - 1) / G : 0;
}
bool batch_prep_fast(int dtype, int ndim, uint32_t B, const BatchArgs& a, const Launch& L);
void batch_prep_generic(int dtype, int ndim, const BatchArgs& a, size_t smem, const Launch& L);
void batch_bound(const Job* jobs, uint32_t n, const Launch& L);
bool batch_predict_fast(int dtype, int ndim, uint32_t B, bool abft, bool enc, const BatchArgs& a, const Launch& L);
void batch_predict_generic(int dtype, int ndim, bool abft, const BatchArgs& a, uint32_t threads, size_t smem,
                           const Launch& L);
void batch_codebook(const Job* jobs, uint32_t n, const Launch& L);
void batch_encode_blocks(int dtype, bool abft, const BatchArgs& a, const Launch& L);
void batch_encode_assemble(int dtype, const BatchArgs& a, const Launch& L);
uint64_t encode_slot_words(const Geo& g);

// Parsed stream header (host side) for the decoder.
struct Hdr {
  Geo g;
  Layout L;
  uint32_t n_live;
  uint64_t n_reg, n_unpred, payload_bytes, total;
  double eb;
  int texp;         // compact encoding: floor(log2 eb), the truncation exponent of unpredictable values
  double cstep[4];  // compact encoding: steps of the coefficient integers
  uint64_t raw_total;  // the stream's size without the lossless stage (== total without it)
};

// Lossless stage. Compression: over the finished stream in w.raw (its layout and size in the
// State), into `out`; sets the State's total to the coded size. Decompression: the stream `s`
// (nbytes) back into `raw` (h.raw_total bytes).
void launch_ll_pack(const Geo& g, const Ws& w, uint8_t* out, uint64_t cap, const Launch& L);
void launch_ll_unpack(const uint8_t* s, uint64_t nbytes, const Hdr& h, uint8_t* raw, State* st, const Launch& L);
// Chunks of a stream whose coded region starts at `from` and whose stream without the stage has
// raw_total bytes.
__host__ __device__ inline uint64_t ll_chunks(uint64_t from, uint64_t raw_total) {
  return raw_total > from ? (raw_total - from + kLLChunk - 1) / kLLChunk : 0;
}
__host__ __device__ inline uint64_t ll_data(uint64_t from, uint64_t nchunks) {
  return align16(from + kLLTable + 4 * nchunks);
}
// Blocks intersecting the box [lo, hi) (padded 3D coordinates) into a dense array of its shape.
void launch_region(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* out, const uint64_t lo[3],
                   const uint64_t hi[3], uint8_t* status, State* st, const Launch& L);
// wave_ws: the two-pass decoder's workspace (wave_decode_ws_bytes), or nullptr (then the one-pass
// kernels decode every shape); the two-pass decoder serves decompression without soft-error
// records only.
void launch_decode(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                   const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                   const Launch& L, uint8_t* wave_ws = nullptr);
bool launch_decode_wave(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status, State* st,
                        uint8_t* wave_ws, const Launch& L);

}  // namespace sdcsz
