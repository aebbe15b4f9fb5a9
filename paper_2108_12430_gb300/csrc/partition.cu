// Placement of independent streams on devices (host only).
//
// Streams share nothing: only each stream's own snapshot update is sequential
// (Methods, "Streaming IaaS"), so a multi-device service shards by stream,
// with no collective on the data path.  The placement balances the streams'
// real-time load (a stream of stride S delivers f_s / S snapshots per second,
// so its load is proportional to 1 / S) under each device's free memory.
#include <algorithm>
#include <numeric>
#include <vector>

#include "gw_internal.h"

extern "C" int gw_partition_streams(int n, const int* stride, const int64_t* bytes, int n_dev, const int64_t* budget,
                                    const int* current, int* device_out, double* load_out) {
  GW_API_BEGIN
  GW_CHECK_ARG(n >= 0 && n_dev >= 1 && (n == 0 || (stride && bytes && device_out)) && budget,
               "NULL argument or bad count");
  for (int i = 0; i < n; ++i) GW_CHECK_ARG(stride[i] >= 1 && bytes[i] >= 0, "stride must be >= 1, bytes >= 0");
  std::vector<double> load(n_dev, 0.0);
  std::vector<int64_t> room(n_dev);
  for (int d = 0; d < n_dev; ++d) room[d] = budget[d];  // < 0: device not available
  std::vector<int> order;
  for (int i = 0; i < n; ++i) {
    device_out[i] = -1;
    // a stream keeps its device while that device is available and has room
    const int c = current ? current[i] : -1;
    if (c >= 0 && c < n_dev && room[c] >= bytes[i]) {
      device_out[i] = c;
      room[c] -= bytes[i];
      load[c] += 1.0 / stride[i];
    } else {
      order.push_back(i);
    }
  }
  // the others in decreasing load (increasing stride), ties by index
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return stride[a] < stride[b]; });
  bool all = true;
  for (int i : order) {
    int best = -1;
    for (int d = 0; d < n_dev; ++d) {
      if (room[d] < bytes[i]) continue;  // also skips unavailable devices (room < 0)
      if (best < 0 || load[d] < load[best]) best = d;
    }
    if (best < 0) {
      all = false;
      continue;
    }
    device_out[i] = best;
    room[best] -= bytes[i];
    load[best] += 1.0 / stride[i];
  }
  if (load_out)
    for (int d = 0; d < n_dev; ++d) load_out[d] = load[d];
  if (!all) throw gw::Error(GW_EBUDGET, "some streams fit on no available device");
  GW_API_END
}
