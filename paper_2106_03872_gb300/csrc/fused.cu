#include "fused.h"

namespace ks {

std::unique_ptr<FusedOps> make_fused_ops(const HostGeometry&, const DevTables<float>&, int, DeviceArena&) {
  return nullptr;
}

}  // namespace ks
