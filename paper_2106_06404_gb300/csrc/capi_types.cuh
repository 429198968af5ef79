// Definitions of the opaque C ABI handles, shared by the entry-point files.
#pragma once
#include <string>
#include <vector>

#include "hierarchy.cuh"

struct msdd_hierarchy {
    msdd::Hierarchy h;
};

struct msdd_band_batch {
    msdd::TileBatch tb;
    int nmax = 0;
    std::vector<int> n;
    msdd::DevBuf<long long> d_src, d_dst;
    msdd::DevBuf<int> d_len;
};

namespace msdd {
// Record the message returned by msdd_last_error() on this thread; returns s.
msdd_status set_last_error(msdd_status s, const std::string& msg);
}  // namespace msdd
