// K5 fast kernels instantiated for double fields in the compact encoding (coefficient integers and
// truncated unpredictable values in the block payloads; see decode.cuh).
#include "decode.cuh"

namespace sdcsz {

void launch_decode_f64_c(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status,
                         const void* original, State* st, bool write, const sdcsz_flip* flips, uint32_t nflips,
                         const Launch& L) {
  kdec::launch_decode_fast_t<double, true>(s, nbytes, h, field, status, original, st, write, flips, nflips, L);
}

}  // namespace sdcsz
