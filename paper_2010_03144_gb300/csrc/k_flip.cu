// Dispatch of K2 by dtype, and the soft-error injectors used by the test entry points.
#include "sdcsz_internal.cuh"

namespace sdcsz {

void launch_predict_f32(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L);
void launch_predict_f64(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L);

void launch_predict(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                    const Launch& L) {
  if (g.dtype == 0) launch_predict_f32(field, g, w, flips, nflips, L);
  else launch_predict_f64(field, g, w, flips, nflips, L);
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
  note_launch();
}

// Soft-error simulation: flip bits of stored codes after their checksums were taken.
__global__ void k_flip_codes(Geo g, Ws w, const sdcsz_flip* flips, uint32_t n) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (flips[t].site != SDCSZ_SITE_CODE || flips[t].block >= g.nb) continue;
    const Box x = block_box(g, flips[t].block);
    if (flips[t].index >= x.P) continue;
    const uint32_t k = (uint32_t)flips[t].index;
    unsigned int* pw = reinterpret_cast<unsigned int*>(w.codes) + pair_index(flips[t].block, g.P, k);
    atomicXor(pw, (1u << (flips[t].bit & 15)) << (16u * (k & 1)));
  }
}

void launch_flip_codes(const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips, const Launch& L) {
  const unsigned grid = (nflips + 255) / 256;
  if (!grid) return;
  k_flip_codes<<<grid, 256, 0, L.stream>>>(g, w, flips, nflips);
  note_launch();
}


bool batch_predict_fast_f32(int ndim, uint32_t B, bool abft, bool enc, const BatchArgs& a, const Launch& L);
bool batch_predict_fast_f64(int ndim, uint32_t B, bool abft, bool enc, const BatchArgs& a, const Launch& L);
void batch_predict_generic_f32(int ndim, bool abft, const BatchArgs& a, uint32_t threads, size_t smem,
                               const Launch& L);
void batch_predict_generic_f64(int ndim, bool abft, const BatchArgs& a, uint32_t threads, size_t smem,
                               const Launch& L);

bool batch_predict_fast(int dtype, int ndim, uint32_t B, bool abft, bool enc, const BatchArgs& a, const Launch& L) {
  return dtype == 0 ? batch_predict_fast_f32(ndim, B, abft, enc, a, L) : batch_predict_fast_f64(ndim, B, abft, enc, a, L);
}

void batch_predict_generic(int dtype, int ndim, bool abft, const BatchArgs& a, uint32_t threads, size_t smem,
                           const Launch& L) {
  if (dtype == 0) batch_predict_generic_f32(ndim, abft, a, threads, smem, L);
  else batch_predict_generic_f64(ndim, abft, a, threads, smem, L);
}

void launch_decode_f32(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                       const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                       const Launch& L);
void launch_decode_f64(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                       const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                       const Launch& L);

void launch_region_f32(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* out, const uint64_t lo[3],
                       const uint64_t hi[3], uint8_t* status, State* st, const Launch& L);
void launch_region_f64(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* out, const uint64_t lo[3],
                       const uint64_t hi[3], uint8_t* status, State* st, const Launch& L);

void launch_region(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* out, const uint64_t lo[3],
                   const uint64_t hi[3], uint8_t* status, State* st, const Launch& L) {
  if (h.g.dtype == 0) launch_region_f32(s, nbytes, h, out, lo, hi, status, st, L);
  else launch_region_f64(s, nbytes, h, out, lo, hi, status, st, L);
}

void launch_decode(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                   const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                   const Launch& L, uint8_t* wave_ws) {
  if (wave_ws && write && !nflips && launch_decode_wave(s, nbytes, h, field, status, st, wave_ws, L)) return;
  if (h.g.dtype == 0) launch_decode_f32(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
  else launch_decode_f64(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
}

}  // namespace sdcsz
