// The host-to-host schedule of lfbp_host_sched.h, exported for the CPU tests
// (TEST INFRASTRUCTURE): each operation as four ints (kind, a, b, wait).
#include <vector>

#include "lfbp_host_sched.h"

extern "C" int sched_run(const long long* zoff, int nz, long long chunk, int memory_order,
                         int* out, int max_ops) {
  std::vector<size_t> z(zoff, zoff + nz + 1);
  const std::vector<lfbp::HostOp> ops = lfbp::host_schedule(z, (size_t)chunk, memory_order != 0);
  if ((int)ops.size() > max_ops) return -1;
  for (size_t i = 0; i < ops.size(); ++i) {
    out[4 * i] = ops[i].kind;
    out[4 * i + 1] = ops[i].a;
    out[4 * i + 2] = ops[i].b;
    out[4 * i + 3] = ops[i].wait;
  }
  return (int)ops.size();
}
