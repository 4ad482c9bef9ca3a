// Float-only instantiation of the libsrhd kernels (SRHD_MIXED_CF): float
// storage and arithmetic, with A of Eq. (transcendental equation) formed by
// error-free products and a compensated float sum (no double arithmetic).
#include "srhd_launch.inl"

namespace srhd {
template struct Launch<PrecMixedCF>;
}
