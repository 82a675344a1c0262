// Register tiers of the X-Drop library (placeholder: routes every unit to the generic tier).
#include "xd_launch.h"

namespace xd {

cudaError_t launch_narrow(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st) {
    (void)P; (void)cfg;
    return launch_route_all_generic(Q, st);
}

cudaError_t launch_wide(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st) {
    (void)P; (void)Q; (void)cfg; (void)st;
    return cudaSuccess;
}

}  // namespace xd
