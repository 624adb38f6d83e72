// NVTX ranges around the library's entry points and build stages. Nsight
// tools show them when one is attached; otherwise a push or pop is a call
// through an empty function pointer. NVTX3 is header-only (it loads a
// tool's injection library with dlopen).
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace flinng {

// A range from construction to end() or destruction, whichever comes first,
// so early error returns keep pushes and pops balanced.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    void end()
    {
        if (open_) nvtxRangePop();
        open_ = false;
    }
    ~TraceRange() { end(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;

private:
    bool open_ = true;
};

}  // namespace flinng
