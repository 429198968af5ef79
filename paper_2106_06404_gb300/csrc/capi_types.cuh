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
// Clear the message, run f and map what it throws to a status with the same
// rules as every other entry point (out of memory -> MSDD_ERR_OOM, a bounded
// wait that gave up -> MSDD_ERR_TIMEOUT, MsddError -> its own status, any
// other failure -> MSDD_ERR_CUDA).  Allocates nothing itself.
msdd_status classified_call(msdd_status (*f)(void*), void* ctx);
// The argument checks of msdd_setup (every field, before any device work):
// MSDD_OK with the effective options in *opt, else the status and a message.
msdd_status check_setup_args(const msdd_mesh* mesh, const msdd_coeff* coeff, const msdd_decomp* decomp,
                             const msdd_spectral* spectral, const msdd_options* options, msdd_options* opt,
                             std::string* msg);
}  // namespace msdd
