// The autotuner's cache of launch choices (tile shapes and schedules per kernel family,
// degree and precision), shared by every handle of the process.
//
// Keys are strings naming the kernel family and the configuration the choice was timed on
// (e.g. "corr3.block nb3 S4"); values are small integers (a block size, a ring depth, a
// grid size in CTAs per 16 SMs).  ridg_autotune writes them after timing the candidates on a
// handle's own state; ridg_create and ridg_batch_create read them.  The cache is loaded once
// from the file named by the environment variable RIDG_TUNE_CACHE (if set) and saved by
// ridg_autotune to the path it is given (one "key value" pair per line).
#pragma once

#include <string>

namespace ridg {

// the tuned value of `key`, or `dflt` if none is recorded
int tune_get(const std::string& key, int dflt);
void tune_put(const std::string& key, int value);
// write the whole cache to `path` (returns false on an I/O error)
bool tune_save(const char* path);
// merge the pairs of `path` into the cache (returns false if it cannot be read)
bool tune_load(const char* path);

}  // namespace ridg
