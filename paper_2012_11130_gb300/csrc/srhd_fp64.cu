// Double-precision instantiation of the libsrhd kernels (SRHD_FP64).
#include "srhd_launch.inl"

namespace srhd {
template struct Launch<PrecFP64>;
}
