// NVTX ranges around the library's stages (histogram accumulation, the iteration and
// its batched forms, energy, prolongation, mesh extraction, the joint solve, the octree
// build, serving steps), so a timeline tool (Nsight Systems, or ncu's NVTX filters)
// shows which call launched which kernels.  NVTX v3 is header-only: with no tool
// attached a push/pop is a check of a null function pointer.  The ranges mark the host
// side of each call; its kernels run asynchronously on the domain's stream.
#pragma once

#include <nvtx3/nvToolsExt.h>

struct TgvNvtxRange {
    explicit TgvNvtxRange(const char* name) { nvtxRangePushA(name); }
    ~TgvNvtxRange() { nvtxRangePop(); }
    TgvNvtxRange(const TgvNvtxRange&) = delete;
    TgvNvtxRange& operator=(const TgvNvtxRange&) = delete;
};
