// launch_shape.cuh -- grid shape of the per-window kernels whose threads each
// walk a run of consecutive windows (window statistics, key seeds).  Long runs
// share a run's setup (a length-m sum) among more windows; short series need
// short runs, or the grid covers a few SMs and the rest stay idle.
#pragma once

namespace mpgb {

// SMs of the current device (1 if the query fails).
int sm_count();

// Run length for `items` windows in each of `groups` independent grids rows,
// blocks of `threads` threads: `run` halved (not below `min_run`) while the
// shorter run still needs no more blocks than there are SMs.
int spread_run(long long items, long long groups, int threads, int run, int min_run);

}  // namespace mpgb
