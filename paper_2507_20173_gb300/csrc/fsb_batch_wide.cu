// fsb_batch_wide.cu -- the batched-schools kernel instantiated for clusters
// of 5 to 8 blocks (fsb_batch.cu instantiates 1 to 4 and holds the host
// side), so the two halves compile in parallel.
#include "fsb_batch_kernel.cuh"

namespace fsb {

const void* batch_kernel_wide(int cluster, int acc, bool var) {
  switch (cluster) {
    case 5: return pick_acc<5>(acc, var);
    case 6: return pick_acc<6>(acc, var);
    case 7: return pick_acc<7>(acc, var);
    case 8: return pick_acc<8>(acc, var);
    default: return nullptr;
  }
}

}  // namespace fsb
