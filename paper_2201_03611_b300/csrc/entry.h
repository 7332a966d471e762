// Instrumentation shared by the extern "C" entry points (host code): an NVTX range named after
// the call, which profilers show and which costs nothing without one attached, and the
// host-side fault injector.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "shine.h"

namespace shine {

struct EntryRange {
    explicit EntryRange(const char* name) { nvtxRangePushA(name); }
    ~EntryRange() { nvtxRangePop(); }
    EntryRange(const EntryRange&) = delete;
    EntryRange& operator=(const EntryRange&) = delete;
};

// SHINE_FAULT_INJECT="<call>=<status>[,<call>=<status>...]" ("*" names every call): each named
// entry point returns that status (1..5) at once, before it reads its arguments or touches the
// GPU, so that callers can exercise their error paths on the host. Unset or empty: no effect.
shine_status injected_fault(const char* name);

}  // namespace shine

#define SHINE_ENTRY(name)                                                      \
    ::shine::EntryRange shine_entry_range_(name);                              \
    if (const shine_status shine_fault_ = ::shine::injected_fault(name)) return shine_fault_
