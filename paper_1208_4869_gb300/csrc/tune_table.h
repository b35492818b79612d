// Launch choices measured on the GPU by paper_1208_4869_gb300/autotune.py
// (rerun it with --write to regenerate this file).  Each entry: for solves
// of precision `dtype` (CCG_C64 / CCG_C128) by `method` on a dense operator
// of order n <= nmax (the first matching entry wins), whether the solve runs
// as one persistent launch (1) or as the kernel-per-step loop (0), and the
// persistent launch's blocks per SM (0: the occupancy limit).
#pragma once

namespace ccg {

struct TuneEntry {
  int dtype, method;
  long long nmax;
  int persistent, pk_blocks;
};

// (no measurements yet: every solve takes the kernel-per-step loop)
static const TuneEntry kTune[] = {
    {-1, -1, 0, 0, 0},
};

}  // namespace ccg
