// zig_internal.h -- declarations shared by the library's translation units.
// Not installed; the public interface is include/zig.h.
#ifndef ZIG_INTERNAL_H
#define ZIG_INTERNAL_H

#include <cstdint>

#include "zig.h"

namespace zig {

// Host construction of both distributions' tables (zig_tables.cpp).
// Returns 0 on success.
int build_host_tables(zig_tables_export* exp_tab, zig_tables_export* nrm_tab);
// The same at i_max = 2^ibits (ibits 8 or 10) in the wide layout.
int build_host_tables_ex(int ibits, zig_tables_ex* exp_tab, zig_tables_ex* nrm_tab);

// Per-box shortcut bounds of the overhang test (zig_tables.cpp): fills
// t->acc52, rej52, acc23, rej23 for box j = 1..L (see zig.h); for the
// exponential acc is at least the always-accept bound of tau.
int box_shortcuts(int dist, zig_tables_ex* t);

// Host tables, built once per process (zig_gen.cu).
const zig_tables_export* host_tables(int dist);

// Tuning cache (zig_tune.cpp): chosen shapes keyed by device name, SM
// count, dist and dtype; JSON Lines load/save return zig_status codes.
void tune_cache_put(const char* device, int sms, int dist, int dtype, const zig_tune_entry& e);
bool tune_cache_get(const char* device, int sms, int dist, int dtype, zig_tune_entry* e);
int tune_cache_load(const char* path);
int tune_cache_save(const char* path);

// zig_gen.cu: whether (V, R, min_blocks) is a compiled candidate for
// dtype, and applying cached choices to every device whose tables are built.
bool tune_shape_known(int dtype, const zig_tune_entry& e);
void tune_apply_loaded();

}  // namespace zig

#endif
