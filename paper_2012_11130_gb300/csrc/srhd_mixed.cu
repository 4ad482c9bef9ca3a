// Mixed-precision instantiation of the libsrhd kernels (SRHD_MIXED): float
// storage and arithmetic, with A of Eq. (transcendental equation) in double.
#include "srhd_launch.inl"

namespace srhd {
template struct Launch<PrecMixed>;
}
