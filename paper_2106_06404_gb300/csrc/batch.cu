// msdd_batch_run: many independent problems set up and solved on one GPU
// (declaration and contract in include/msdd.h).
//
// A host work queue hands the problems out largest first (cost: the sum over
// fine subdomains of n (b + 1), the band size that the factorisations and
// every band solve of the subspace iteration scale with) to worker threads.
// Each worker owns non-blocking streams and runs set-up and PCG of one
// problem after the other, so kernels of different problems run side by
// side on the GPU instead of one small problem leaving most SMs idle.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <thread>

#include "capi_types.cuh"

namespace {

// the element reference matrices (constant memory) are shared by all
// problems of a batch: their elements must have the same shape
bool same_element_shape(const msdd_mesh& a, const msdd_mesh& b) {
    if (a.dim != b.dim) return false;
    // equal shape <=> the element edge ratios agree: n[d] n[0]' == n[0] n[d]'
    for (int d = 1; d < a.dim; ++d)
        if ((long long)a.n[d] * b.n[0] != (long long)b.n[d] * a.n[0]) return false;
    return true;
}

double problem_cost(const msdd_mesh& mesh, const msdd_decomp& dec) {
    msdd_coeff none{0, nullptr};
    const msdd::Geom g = msdd::make_geom(mesh, none);
    double c = 0.0;
    for (const msdd::ProbBox& b : msdd::make_fine_boxes(g, dec)) {
        long long w[3] = {1, 1, 1}, n = 1;
        for (int d = 0; d < mesh.dim; ++d) {
            w[d] = b.nhi[d] - b.nlo[d] + 1;
            n *= w[d];
        }
        const long long bw = mesh.dim == 3 ? w[0] * w[1] + w[0] + 1 : w[0] + 1;
        c += (double)n * (double)(bw + 1);
    }
    return c;
}

msdd_status status_of(const std::exception_ptr& ep, std::string* msg) {
    try {
        std::rethrow_exception(ep);
    } catch (const msdd::MsddError& e) {
        *msg = e.what();
        return e.status;
    } catch (const msdd::CudaError& e) {
        *msg = e.what();
        return std::string(e.what()).find("out of memory") != std::string::npos ? MSDD_ERR_OOM : MSDD_ERR_CUDA;
    } catch (const msdd::WaitTimeout& e) {
        *msg = e.what();
        return MSDD_ERR_TIMEOUT;
    } catch (const std::bad_alloc&) {
        *msg = "host allocation failed";
        return MSDD_ERR_OOM;
    } catch (const std::exception& e) {
        *msg = e.what();
        return MSDD_ERR_CUDA;
    }
}

}  // namespace

extern "C" msdd_status msdd_batch_run(int nprob, const msdd_mesh* meshes, const msdd_coeff* coeffs,
                                      const msdd_decomp* decomps, const msdd_spectral* spectral,
                                      const msdd_options* options, const double* const* b, double tol, int maxit,
                                      double* const* x, int nworkers, int* iterations, double* rel_residual,
                                      int* status, double* setup_ms, double* solve_ms) {
    if (nprob < 1 || !meshes || !coeffs || !decomps || !spectral || !b || !x || !status || nworkers < 1 ||
        !(tol > 0.0) || maxit < 1)
        return msdd::set_last_error(MSDD_ERR_INVALID_ARG, "invalid batch arguments");
    // every problem's arguments are checked before any device work
    std::vector<msdd_options> opts(nprob);
    for (int p = 0; p < nprob; ++p) {
        std::string msg;
        const msdd_status st =
            msdd::check_setup_args(&meshes[p], &coeffs[p], &decomps[p], spectral, options, &opts[p], &msg);
        if (st == MSDD_OK && (!b[p] || !x[p])) return msdd::set_last_error(MSDD_ERR_INVALID_ARG, "NULL b or x");
        if (st != MSDD_OK) return msdd::set_last_error(st, "problem " + std::to_string(p) + ": " + msg);
        if (!same_element_shape(meshes[0], meshes[p]))
            return msdd::set_last_error(MSDD_ERR_UNSUPPORTED,
                                        "problem " + std::to_string(p) + ": the problems of a batch must have "
                                        "elements of one shape");
    }
    // the shared reference matrices, once for all problems (every set-up
    // then finds them in place and uploads nothing)
    try {
        msdd::upload_reference(msdd::make_geom(meshes[0], coeffs[0]));
    } catch (...) {
        std::string msg;
        const msdd_status st = status_of(std::current_exception(), &msg);
        return msdd::set_last_error(st, msg);
    }
    std::vector<int> order(nprob);
    std::vector<double> cost(nprob);
    for (int p = 0; p < nprob; ++p) cost[p] = problem_cost(meshes[p], decomps[p]);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });

    std::atomic<int> next{0};
    std::vector<std::string> msgs(nprob);
    const int W = std::min(nworkers, nprob);
    auto worker = [&]() {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= nprob) break;
            const int p = order[k];
            if (!s) {
                status[p] = MSDD_ERR_CUDA;
                msgs[p] = "stream creation failed";
                continue;
            }
            try {
                msdd_hierarchy H;
                H.h.opt = opts[p];
                H.h.opt.stream = s;
                H.h.spec = *spectral;
                H.h.dec = decomps[p];
                H.h.st = s;
                H.h.setup(meshes[p], coeffs[p]);
                double rr = 0.0;
                const int it = H.h.solve(b[p], tol, maxit, x[p], &rr);
                if (iterations) iterations[p] = it < 0 ? -it : it;
                if (rel_residual) rel_residual[p] = rr;
                if (setup_ms) setup_ms[p] = H.h.stats.setup_ms;
                if (solve_ms) solve_ms[p] = H.h.stats.solve_ms;
                status[p] = it < 0 ? MSDD_ERR_NO_CONVERGENCE : MSDD_OK;
                if (H.h.stats.eig_unconverged[H.h.L] || (H.h.levels == 3 && H.h.stats.eig_unconverged[1]))
                    status[p] = status[p] == MSDD_OK ? MSDD_ERR_EIG_NO_CONVERGENCE : status[p];
            } catch (...) {
                status[p] = status_of(std::current_exception(), &msgs[p]);
            }
            // the hierarchy is gone and its internal streams were synchronised
            // by its destructor; once this worker's stream is idle too, the
            // blocks it released can serve the next problems
            if (cudaStreamSynchronize(s) == cudaSuccess) msdd::dev_cache_collect_thread();
        }
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        msdd::kernel_launch_flush();
    };
    std::vector<std::thread> threads;
    threads.reserve(W);
    for (int w = 0; w < W; ++w) threads.emplace_back(worker);
    for (auto& t : threads) t.join();
    msdd::dev_cache_collect();
    for (int k = 0; k < nprob; ++k) {
        const int p = order[k];
        if (status[p] != MSDD_OK)
            return msdd::set_last_error((msdd_status)status[p],
                                        "problem " + std::to_string(p) + ": " +
                                            (msgs[p].empty() ? std::string("see its status") : msgs[p]));
    }
    return msdd::set_last_error(MSDD_OK, "");
}
