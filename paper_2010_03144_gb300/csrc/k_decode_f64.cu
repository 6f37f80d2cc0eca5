// K5 kernels instantiated for double fields in the raw encoding, the generic kernel and region
// decompression (see decode.cuh).
#include "decode.cuh"

namespace sdcsz {

void launch_decode_f64_c(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                         const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                         const Launch& L);

// Shapes with a fast path take the fast kernels of their encoding (the compact encoding's in
// k_decode_f64c.cu); other shapes the generic kernel.
void launch_decode_f64(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                      const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                      const Launch& L) {
  if (!kdec::has_fast<double>(h.g))
    kdec::launch_decode_generic_t<double>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
  else if (h.g.enc)
    launch_decode_f64_c(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
  else
    kdec::launch_decode_fast_t<double, false>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
}

void launch_region_f64(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* out, const uint64_t lo[3],
                        const uint64_t hi[3], uint8_t* status, State* st, const Launch& L) {
  kdec::Region r;
  for (int a = 0; a < 3; ++a) {
    r.lo[a] = lo[a];
    r.hi[a] = hi[a];
    r.c0[a] = lo[a] / h.g.B[a];
    r.nc[a] = hi[a] > lo[a] ? (hi[a] - 1) / h.g.B[a] - r.c0[a] + 1 : 0;
  }
  kdec::launch_region_t<double>(s, nbytes, h, out, r, status, st, L);
}

}  // namespace sdcsz
