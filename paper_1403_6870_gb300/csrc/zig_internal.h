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

// Host tables, built once per process (zig_gen.cu).
const zig_tables_export* host_tables(int dist);

}  // namespace zig

#endif
