// Block-per-box schedule for batches of small boxes (placeholder until the
// persistent kernel lands).
#include "md_device.cuh"

namespace mdk {

bool box_schedule_fits(const Engine&) { return false; }

int launch_box_steps(Engine&, int, cudaStream_t) { return MD_ERR_UNSUPPORTED; }

}  // namespace mdk
