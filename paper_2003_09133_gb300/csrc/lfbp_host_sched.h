// Order of the copies and maps of the host-to-host path (host code only).
//
// The path moves H from host memory to the device in fixed byte ranges
// ("chunks"), maps each depth once every chunk it overlaps has arrived, and
// copies a chunk of H' back once every depth overlapping it is mapped.  Copies
// in and copies back run at the same time on two streams, so a step costs about
// the time of both directions at once plus a fill (the bytes that must arrive
// before the first map) and a drain (what is still to go back after the last
// chunk has arrived).  Both are set by the depths processed first and last.
// The default order is the memory order.  The other order is a rotation of it
// that starts at the smallest depth: up to the last depth and round to the one
// before the start, or down to the first and round to the one after it,
// whichever ends on the smaller depth (adjacent depths stay adjacent, except
// at the wrap).  On the 41-depth highres workload with 64 MiB chunks it cuts
// the fill from 256 to 64 MiB and the drain from 220 to 192 MiB, but measured
// slower (24.09 against 23.83 ms per step): bytes moved in one direction
// alone go faster than while both directions share the link, so the fill and
// drain cost less than their size suggests.
#pragma once

#include <cstddef>
#include <vector>

namespace lfbp {

struct HostOp {
  enum Kind { kIn = 0, kMap = 1, kOut = 2 };
  int kind;
  int a, b;  // kIn / kOut: chunk a; kMap: depths [a, b)
  int wait;  // kMap: the chunk whose arrival it waits for (the last one issued that it needs)
};

// Depth order: with `memory_order` the depths in memory order, else the
// rotation described above.  Empty depths are left out.
inline std::vector<int> host_depth_order(const std::vector<size_t>& zoff, bool memory_order) {
  const int nz = (int)zoff.size() - 1;
  std::vector<int> nonempty;
  for (int z = 0; z < nz; ++z)
    if (zoff[z + 1] > zoff[z]) nonempty.push_back(z);
  if (memory_order || nonempty.size() < 3) return nonempty;
  const int n = (int)nonempty.size();
  auto size = [&](int i) { return zoff[nonempty[i] + 1] - zoff[nonempty[i]]; };
  int m = 0;  // the smallest depth (the first of equals)
  for (int i = 1; i < n; ++i)
    if (size(i) < size(m)) m = i;
  // upwards the last depth is m-1 (wrapping), downwards m+1
  const int last_up = (m + n - 1) % n, last_down = (m + 1) % n;
  const bool up = size(last_up) <= size(last_down);
  std::vector<int> order;
  for (int j = 0; j < n; ++j) order.push_back(nonempty[up ? (m + j) % n : (m - j + n) % n]);
  return order;
}

// The operations in issue order for depths with byte offsets zoff (Nz + 1
// entries, non-decreasing) and chunks of `chunk` bytes.  Consecutive maps of
// adjacent depths whose chunks have all arrived by the same wait are merged
// into one range.
inline std::vector<HostOp> host_schedule(const std::vector<size_t>& zoff, size_t chunk,
                                         bool memory_order) {
  std::vector<HostOp> ops;
  const size_t bytes = zoff.back();
  if (bytes == 0 || chunk == 0) return ops;
  const int nch = (int)((bytes + chunk - 1) / chunk);
  const int nz = (int)zoff.size() - 1;
  // pending[k]: depths overlapping chunk k not yet mapped
  std::vector<int> pending(nch, 0), issue_pos(nch, -1);
  for (int z = 0; z < nz; ++z) {
    if (zoff[z + 1] == zoff[z]) continue;
    for (size_t k = zoff[z] / chunk; k <= (zoff[z + 1] - 1) / chunk; ++k) ++pending[k];
  }
  int issued = 0;
  for (int z : host_depth_order(zoff, memory_order)) {
    const int k0 = (int)(zoff[z] / chunk), k1 = (int)((zoff[z + 1] - 1) / chunk);
    int wait = -1;  // the chunk of this depth issued last
    for (int k = k0; k <= k1; ++k) {
      if (issue_pos[k] < 0) {
        issue_pos[k] = issued++;
        ops.push_back(HostOp{HostOp::kIn, k, k + 1, -1});
      }
      if (wait < 0 || issue_pos[k] > issue_pos[wait]) wait = k;
    }
    // merge with the previous map when its wait covers this depth's chunks
    // (copies in complete in issue order) and the depth ranges touch; a copy
    // back issued in between ends the previous map
    HostOp& prev = ops.back();
    if (prev.kind == HostOp::kMap && issue_pos[wait] <= issue_pos[prev.wait] &&
        (prev.b == z || prev.a == z + 1)) {
      prev.a = prev.a < z ? prev.a : z;
      prev.b = prev.b > z + 1 ? prev.b : z + 1;
    } else {
      ops.push_back(HostOp{HostOp::kMap, z, z + 1, wait});
    }
    // chunks whose every depth is now mapped go back: those of this depth
    // only (no other chunk changes) -- issued after the map above is released
    std::vector<HostOp> outs;
    for (int k = k0; k <= k1; ++k)
      if (--pending[k] == 0) outs.push_back(HostOp{HostOp::kOut, k, k + 1, -1});
    ops.insert(ops.end(), outs.begin(), outs.end());
  }
  return ops;
}

}  // namespace lfbp
