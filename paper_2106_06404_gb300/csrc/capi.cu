// C ABI of the msdd library (declarations and contracts in include/msdd.h).
#include <algorithm>
#include <atomic>
#include <functional>
#include <queue>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "capi_types.cuh"
#include "warmstart.cuh"

namespace msdd {
// launches counted per host thread (graph capture subtracts what it captured);
// worker threads of a batch add theirs to the process total when they end
namespace {
std::atomic<long long> g_launch_total{0};
thread_local long long t_launches = 0;
}  // namespace
long long& kernel_launch_counter() { return t_launches; }
void kernel_launch_flush() {
    g_launch_total += t_launches;
    t_launches = 0;
}
long long kernel_launch_total() { return g_launch_total.load() + t_launches; }
}  // namespace msdd

namespace {

thread_local std::string g_last_error;

msdd_status fail(msdd_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

}  // namespace

msdd_status msdd::set_last_error(msdd_status s, const std::string& msg) { return fail(s, msg); }

namespace {

template <class F>
msdd_status guarded_call(F&& f) {
    try {
        g_last_error.clear();
        return f();
    } catch (const msdd::MsddError& e) {
        return fail(e.status, e.what());
    } catch (const msdd::CudaError& e) {
        std::string m = e.what();
        if (m.find("out of memory") != std::string::npos) return fail(MSDD_ERR_OOM, m);
        return fail(MSDD_ERR_CUDA, m);
    } catch (const msdd::WaitTimeout& e) {
        return fail(MSDD_ERR_TIMEOUT, e.what());
    } catch (const std::bad_alloc&) {
        return fail(MSDD_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(MSDD_ERR_CUDA, e.what());
    }
}

}  // namespace

msdd_status msdd::classified_call(msdd_status (*f)(void*), void* ctx) {
    return guarded_call([&]() -> msdd_status { return f(ctx); });
}

namespace {

// every entry point: blocks released during the call become reusable
// (device synchronised once, only if the call released any)
template <class F>
msdd_status guarded(F&& f) {
    const msdd_status st = guarded_call(std::forward<F>(f));
    msdd::dev_cache_collect();
    return st;
}

bool mesh_ok(const msdd_mesh* m) {
    if (!m || (m->dim != 2 && m->dim != 3)) return false;
    for (int d = 0; d < m->dim; ++d)
        if (m->n[d] < 1 || m->n[d] > (1 << 20)) return false;
    unsigned mask = m->dim == 2 ? 0xFu : 0x3Fu;
    if ((m->dirichlet_faces & mask) == 0) return false;
    if (m->dirichlet_faces & ~mask) return false;
    for (int d = 0; d < m->dim; ++d)
        if (((m->dirichlet_faces >> (2 * d)) & 3u) == 3u && m->n[d] < 2) return false;
    return true;
}

long long unknowns_of(const msdd_mesh* m) {
    long long n = 1;
    for (int d = 0; d < m->dim; ++d) {
        int lo = (m->dirichlet_faces >> (2 * d)) & 1 ? 1 : 0;
        int hi = (m->dirichlet_faces >> (2 * d + 1)) & 1 ? m->n[d] - 1 : m->n[d];
        n *= (hi - lo + 1);
    }
    return n;
}

bool decomp_parts_ok(const msdd_mesh* mesh, const msdd_decomp* dec) {
    if (!dec || dec->overlap < 1) return false;
    for (int d = 0; d < mesh->dim; ++d)
        if (dec->parts[d] < 1 || dec->parts[d] > mesh->n[d]) return false;
    return true;
}

// fine boxes of a 2D scalar-coefficient problem for the warm-start calls
std::vector<msdd::ProbBox> warm_boxes(const msdd_mesh* mesh, const msdd_decomp* decomp, msdd::Geom& g) {
    msdd_coeff none{0, nullptr};
    g = msdd::make_geom(*mesh, none);
    return msdd::make_fine_boxes(g, *decomp);
}

}  // namespace

msdd_status msdd::check_setup_args(const msdd_mesh* mesh, const msdd_coeff* coeff, const msdd_decomp* decomp,
                                   const msdd_spectral* spectral, const msdd_options* options, msdd_options* opt_out,
                                   std::string* msg) {
    auto bad = [&](msdd_status st, const char* m) {
        *msg = m;
        return st;
    };
    if (!mesh_ok(mesh)) return bad(MSDD_ERR_INVALID_ARG, "invalid mesh (dim, sizes or Dirichlet faces)");
    if (!coeff || !coeff->data || (coeff->kind != 0 && coeff->kind != 1))
        return bad(MSDD_ERR_INVALID_ARG, "invalid coefficient");
    if (!decomp || !spectral) return bad(MSDD_ERR_INVALID_ARG, "decomposition or spectral options NULL");
    if (decomp->levels < 2) return bad(MSDD_ERR_INVALID_ARG, "levels must be >= 2");
    if (decomp->levels > 3) return bad(MSDD_ERR_UNSUPPORTED, "this build supports 2 or 3 levels");
    if (decomp->overlap < 1) return bad(MSDD_ERR_INVALID_ARG, "overlap must be >= 1 (partition of unity)");
    for (int d = 0; d < mesh->dim; ++d) {
        if (decomp->parts[d] < 1 || decomp->parts[d] > mesh->n[d])
            return bad(MSDD_ERR_INVALID_ARG, "parts must be in 1..n per axis");
        if (decomp->levels == 3 && decomp->group[d] < 1) return bad(MSDD_ERR_INVALID_ARG, "group must be >= 1 per axis");
    }
    if (spectral->nev_max < 1 || spectral->nev_max > 24 || !(spectral->eta > 0.0))
        return bad(MSDD_ERR_INVALID_ARG, "nev_max must be in 1..24 and eta > 0");
    if (spectral->blf < 0 || spectral->blf > 3) return bad(MSDD_ERR_INVALID_ARG, "blf must be 1, 2 or 3");
    msdd_options opt;
    msdd_default_options(&opt);
    if (options) opt = *options;
    if (opt.precision != 0 && opt.precision != 1) return bad(MSDD_ERR_INVALID_ARG, "precision must be 0 or 1");
    if (opt.block_p < 0 || opt.block_p > msdd::PMAX) return bad(MSDD_ERR_INVALID_ARG, "block_p out of range");
    if (opt.block_p > 0 && opt.block_p <= spectral->nev_max)
        return bad(MSDD_ERR_INVALID_ARG, "block_p must exceed nev_max");
    if (!(opt.sigma > 0.0) || !(opt.eig_tol > 0.0) || opt.eig_maxit < 1 || !(opt.reg_tol < 1.0) ||
        opt.fp32_start_iters < 0 || opt.fp32_start_iters > 1000)
        return bad(MSDD_ERR_INVALID_ARG, "invalid eigensolver options");
    if (opt.warm_start && (opt.warm_cols < 1 || opt.warm_cols > msdd::PMAX))
        return bad(MSDD_ERR_INVALID_ARG, "warm_cols must be in 1..32 with warm_start");
    *opt_out = opt;
    return MSDD_OK;
}

extern "C" {

const char* msdd_last_error(void) { return g_last_error.c_str(); }

msdd_status msdd_default_options(msdd_options* opt) {
    if (!opt) return fail(MSDD_ERR_INVALID_ARG, "options pointer is NULL");
    opt->precision = 0;
    opt->block_p = 0;
    opt->eig_maxit = 200;
    opt->sigma = 1e-2;
    opt->eig_tol = 1e-6;
    opt->reg_tol = -1.0;            // automatic: 1e-10 in 2D, 1e-6 in 3D
    opt->seed = 12345;
    opt->stream = nullptr;
    opt->profile = 0;
    opt->fp32_start_iters = 20;
    opt->warm_start = nullptr;
    opt->warm_cols = 0;
    return MSDD_OK;
}

long long msdd_num_unknowns(const msdd_mesh* mesh) {
    if (!mesh_ok(mesh)) return -1;
    return unknowns_of(mesh);
}

msdd_status msdd_setup(const msdd_mesh* mesh, const msdd_coeff* coeff, const msdd_decomp* decomp,
                       const msdd_spectral* spectral, const msdd_options* options, msdd_hierarchy** out) {
    return guarded([&]() -> msdd_status {
        if (!out) return fail(MSDD_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        msdd_options opt;
        std::string msg;
        const msdd_status chk = msdd::check_setup_args(mesh, coeff, decomp, spectral, options, &opt, &msg);
        if (chk != MSDD_OK) return fail(chk, msg);
        msdd_hierarchy* H = new msdd_hierarchy();
        H->h.opt = opt;
        H->h.spec = *spectral;
        H->h.dec = *decomp;
        H->h.st = (cudaStream_t)opt.stream;
        try {
            H->h.setup(*mesh, *coeff);
        } catch (...) {
            delete H;
            throw;
        }
        *out = H;
        if (H->h.stats.eig_unconverged[H->h.L] || (H->h.levels == 3 && H->h.stats.eig_unconverged[1])) {
            g_last_error = "subspace iteration reached eig_maxit on some subdomains (hierarchy kept)";
            return MSDD_ERR_EIG_NO_CONVERGENCE;
        }
        return MSDD_OK;
    });
}

msdd_status msdd_solve(msdd_hierarchy* h, const double* b, double tol, int maxit, double* x, int* iterations,
                       double* rel_residual) {
    return guarded([&]() -> msdd_status {
        if (!h || !b || !x) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        if (!(tol > 0.0) || maxit < 1) return fail(MSDD_ERR_INVALID_ARG, "tol must be > 0 and maxit >= 1");
        int it = h->h.solve(b, tol, maxit, x, rel_residual);
        if (iterations) *iterations = it < 0 ? -it : it;
        if (it < 0) return fail(MSDD_ERR_NO_CONVERGENCE, "CG reached maxit");
        return MSDD_OK;
    });
}

msdd_status msdd_solve_host(msdd_hierarchy* h, const double* b, double tol, int maxit, double* x, int* iterations,
                            double* rel_residual) {
    return guarded([&]() -> msdd_status {
        if (!h || !b || !x) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        long long n = h->h.nun;
        msdd::DevBuf<double> db(n), dx(n);
        cudaStream_t st = h->h.st;
        MSDD_CUDA(cudaMemcpyAsync(db.p, b, n * sizeof(double), cudaMemcpyHostToDevice, st));
        msdd_status s = msdd_solve(h, db.p, tol, maxit, dx.p, iterations, rel_residual);
        if (s != MSDD_OK && s != MSDD_ERR_NO_CONVERGENCE) return s;
        MSDD_CUDA(cudaMemcpyAsync(x, dx.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        MSDD_CUDA(cudaStreamSynchronize(st));
        return s;
    });
}

msdd_status msdd_apply_preconditioner(msdd_hierarchy* h, const double* r, double* z) {
    return guarded([&]() -> msdd_status {
        if (!h || !r || !z) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        h->h.apply_prec(r, z, nullptr);
        MSDD_CUDA(cudaStreamSynchronize(h->h.st));
        return MSDD_OK;
    });
}

msdd_status msdd_apply_hybrid_preconditioner(msdd_hierarchy* h, const double* r, double* z) {
    return guarded([&]() -> msdd_status {
        if (!h || !r || !z) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        h->h.apply_hybrid(r, z);
        MSDD_CUDA(cudaStreamSynchronize(h->h.st));
        return MSDD_OK;
    });
}

msdd_status msdd_solve_gmres(msdd_hierarchy* h, const double* b, double tol, int restart, int maxit, double* x,
                             int* iterations, double* rel_residual) {
    return guarded([&]() -> msdd_status {
        if (!h || !b || !x) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        if (!(tol > 0.0) || maxit < 1 || restart < 1 || restart > 1000)
            return fail(MSDD_ERR_INVALID_ARG, "tol must be > 0, maxit >= 1 and restart in 1..1000");
        int it = h->h.solve_gmres(b, tol, restart, maxit, x, rel_residual);
        if (iterations) *iterations = it < 0 ? -it : it;
        if (it < 0) return fail(MSDD_ERR_NO_CONVERGENCE, "GMRES reached maxit");
        return MSDD_OK;
    });
}

msdd_status msdd_apply_operator(msdd_hierarchy* h, const double* x, double* y) {
    return guarded([&]() -> msdd_status {
        if (!h || !x || !y) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        msdd::upload_reference(h->h.g);            // this hierarchy's element shape
        msdd::apply_global(h->h.g, x, y, h->h.st);
        MSDD_CUDA(cudaStreamSynchronize(h->h.st));
        return MSDD_OK;
    });
}

msdd_status msdd_assemble_rhs(const msdd_mesh* mesh, double f, double* b, void* stream) {
    return guarded([&]() -> msdd_status {
        if (!mesh_ok(mesh) || !b) return fail(MSDD_ERR_INVALID_ARG, "invalid mesh or NULL b");
        msdd::Geom g{};
        g.dim = mesh->dim;
        for (int d = 0; d < 3; ++d) {
            g.n[d] = d < mesh->dim ? mesh->n[d] : 1;
            if (d < mesh->dim) {
                g.ulo[d] = (mesh->dirichlet_faces >> (2 * d)) & 1 ? 1 : 0;
                g.uhi[d] = (mesh->dirichlet_faces >> (2 * d + 1)) & 1 ? g.n[d] - 1 : g.n[d];
            }
            g.ushape[d] = g.uhi[d] - g.ulo[d] + 1;
        }
        msdd::load_vector(g, f, b, (cudaStream_t)stream);
        MSDD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return MSDD_OK;
    });
}

msdd_status msdd_get_stats(const msdd_hierarchy* h, msdd_stats* out) {
    if (!h || !out) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
    *out = h->h.stats;
    return MSDD_OK;
}

msdd_status msdd_get_eigenvalues(const msdd_hierarchy* h, int level, int subdomain, double* out, int cap, int* count,
                                 int* selected) {
    return guarded([&]() -> msdd_status {
        if (!h || !out || cap < 0) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        const msdd::GevpBatch* gb = nullptr;
        if (level == h->h.L) gb = &h->h.fge;
        else if (h->h.levels == 3 && level == 1) gb = &h->h.mge;
        else return fail(MSDD_ERR_INVALID_ARG, "level has no eigenproblems");
        if (subdomain < 0 || subdomain >= gb->P) return fail(MSDD_ERR_INVALID_ARG, "subdomain out of range");
        int p = gb->p[subdomain];
        std::vector<double> th(msdd::PMAX);
        MSDD_CUDA(cudaMemcpy(th.data(), gb->theta.p + (size_t)subdomain * msdd::PMAX, msdd::PMAX * sizeof(double),
                             cudaMemcpyDeviceToHost));
        int mval = 0;
        MSDD_CUDA(cudaMemcpy(&mval, gb->m.p + subdomain, sizeof(int), cudaMemcpyDeviceToHost));
        for (int k = 0; k < std::min(cap, p); ++k) out[k] = th[k];
        if (count) *count = p;
        if (selected) *selected = mval;
        return MSDD_OK;
    });
}

msdd_status msdd_get_eigen_residuals(const msdd_hierarchy* h, int level, int subdomain, double* out, int cap,
                                     int* converged) {
    return guarded([&]() -> msdd_status {
        if (!h || !out || cap < 0) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        const msdd::GevpBatch* gb = nullptr;
        if (level == h->h.L) gb = &h->h.fge;
        else if (h->h.levels == 3 && level == 1) gb = &h->h.mge;
        else return fail(MSDD_ERR_INVALID_ARG, "level has no eigenproblems");
        if (subdomain < 0 || subdomain >= gb->P) return fail(MSDD_ERR_INVALID_ARG, "subdomain out of range");
        std::vector<double> r(msdd::PMAX);
        MSDD_CUDA(cudaMemcpy(r.data(), gb->res.p + (size_t)subdomain * msdd::PMAX, msdd::PMAX * sizeof(double),
                             cudaMemcpyDeviceToHost));
        int dn = 0;
        MSDD_CUDA(cudaMemcpy(&dn, gb->done.p + subdomain, sizeof(int), cudaMemcpyDeviceToHost));
        for (int k = 0; k < std::min(cap, gb->p[subdomain]); ++k) out[k] = r[k];
        if (converged) *converged = (dn == 1 || dn == 3) ? 1 : 0;
        return MSDD_OK;
    });
}

msdd_status msdd_get_fine_basis(const msdd_hierarchy* h, int subdomain, double* out, long long cap, int* m_out) {
    return guarded([&]() -> msdd_status {
        if (!h || !out) return fail(MSDD_ERR_INVALID_ARG, "NULL argument");
        const msdd::Hierarchy& H = h->h;
        if (subdomain < 0 || subdomain >= H.Pf) return fail(MSDD_ERR_INVALID_ARG, "subdomain out of range");
        int m = H.fm[subdomain];
        if (m_out) *m_out = m;
        if (cap < H.nun * (long long)m) return fail(MSDD_ERR_INVALID_ARG, "output too small (n * m doubles)");
        const msdd::ProbBox& b = H.fboxes[subdomain];
        int nd = msdd::box_size(b.dlo, b.dhi, H.g.dim);
        std::vector<double> blk((size_t)nd * H.ldphi);
        MSDD_CUDA(cudaMemcpy(blk.data(), H.Phi.p + H.phioff[subdomain], blk.size() * sizeof(double),
                             cudaMemcpyDeviceToHost));
        std::fill(out, out + H.nun * m, 0.0);
        for (int r = 0; r < nd; ++r) {
            int x[3];
            msdd::box_coords(r, b.dlo, b.dhi, H.g.dim, x);
            long long u = msdd::unknown_index(H.g, x);
            for (int k = 0; k < m; ++k) out[u * m + k] = blk[(size_t)r * H.ldphi + k];
        }
        return MSDD_OK;
    });
}

void msdd_destroy(msdd_hierarchy* h) {
    delete h;
    msdd::dev_cache_collect();
}

msdd_status msdd_release_cache(void) {
    return guarded([&]() -> msdd_status {
        msdd::dev_cache_trim();
        return MSDD_OK;
    });
}

long long msdd_cached_bytes(void) { return (long long)msdd::dev_cache_bytes(); }

long long msdd_kernel_launches(void) { return msdd::kernel_launch_total(); }

msdd_status msdd_band_factor(int batch, const int* n, int nmax, int bw, const double* A, int precision,
                             double reg_tol, void* stream, msdd_band_batch** out, int* status) {
    return guarded([&]() -> msdd_status {
        if (!out) return fail(MSDD_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        if (batch < 1 || !n || !A || nmax < 1 || bw < 0 || (precision != 0 && precision != 1) || reg_tol < 0.0)
            return fail(MSDD_ERR_INVALID_ARG, "invalid band batch arguments");
        std::vector<int> nv(n, n + batch);
        for (int v : nv)
            if (v < 1 || v > nmax) return fail(MSDD_ERR_INVALID_ARG, "n[i] must be in 1..nmax");
        cudaStream_t st = (cudaStream_t)stream;
        msdd_band_batch* bb = new msdd_band_batch();
        try {
            bb->nmax = nmax;
            bb->n = nv;
            std::vector<int> bws(batch, bw);
            bb->tb.layout(nv, bws, precision, st);
            std::vector<long long> so(batch);
            std::vector<int> ld(batch, nmax);
            for (int i = 0; i < batch; ++i) so[i] = (long long)i * nmax * nmax;
            msdd::DevBuf<long long> d_so;
            d_so.upload(so, st);
            msdd::DevBuf<int> d_ld;
            d_ld.upload(ld, st);
            // only the lower band |r - c| <= bw is copied into the tiles
            msdd::tile_from_dense(bb->tb, A, d_so.p, d_ld.p, st);
            msdd::tile_factor(bb->tb, reg_tol, st);
            std::vector<int> stv = bb->tb.d_status.download(st);
            bool bad = false;
            for (int i = 0; i < batch; ++i) {
                if (status) status[i] = stv[i];
                bad = bad || stv[i] != 0;
            }
            MSDD_CUDA(cudaStreamSynchronize(st));
            if (bad) {
                delete bb;
                return fail(MSDD_ERR_NOT_SPD, "non-positive pivot (see status)");
            }
        } catch (...) {
            delete bb;
            throw;
        }
        *out = bb;
        return MSDD_OK;
    });
}

msdd_status msdd_band_solve(const msdd_band_batch* bb, int nrhs, double* X, void* stream) {
    return guarded([&]() -> msdd_status {
        if (!bb || !X || nrhs < 1 || nrhs > msdd::PMAX) return fail(MSDD_ERR_INVALID_ARG, "invalid band solve arguments");
        cudaStream_t st = (cudaStream_t)stream;
        const int P = bb->tb.P;
        msdd::DevBuf<double> stage((size_t)bb->tb.total_rows * nrhs);
        stage.zero(st);
        std::vector<long long> so(P), dof(P);
        std::vector<int> len(P);
        int maxlen = 0;
        for (int i = 0; i < P; ++i) {
            so[i] = (long long)i * bb->nmax * nrhs;
            dof[i] = bb->tb.roff[i] * nrhs;
            len[i] = bb->n[i] * nrhs;
            maxlen = std::max(maxlen, len[i]);
        }
        msdd::DevBuf<long long> d_so, d_do;
        msdd::DevBuf<int> d_len;
        d_so.upload(so, st);
        d_do.upload(dof, st);
        d_len.upload(len, st);
        msdd::segment_copy(d_so.p, d_do.p, d_len.p, P, maxlen, X, stage.p, 0, nullptr, st);
        msdd::tile_solve(bb->tb, stage.p, nrhs, nrhs, nullptr, st);
        msdd::segment_copy(d_do.p, d_so.p, d_len.p, P, maxlen, stage.p, X, 0, nullptr, st);
        MSDD_CUDA(cudaStreamSynchronize(st));
        msdd::tile_check_waits();
        return MSDD_OK;
    });
}

void msdd_band_destroy(msdd_band_batch* bb) {
    delete bb;
    msdd::dev_cache_collect();
}

// ---- learned warm start
msdd_status msdd_batch_plan(int nprob, const msdd_mesh* meshes, const msdd_decomp* decomps, int nworkers,
                            int* items, double* cost, long long cap, long long* count, double* makespan,
                            double* lower_bound) {
    return guarded_call([&]() -> msdd_status {
        if (nprob < 1 || !meshes || !decomps || nworkers < 1)
            return fail(MSDD_ERR_INVALID_ARG, "nprob >= 1, meshes, decomps and nworkers >= 1 are required");
        struct Item {
            double c;
            int p, s;
        };
        std::vector<Item> all;
        for (int p = 0; p < nprob; ++p) {
            if (!mesh_ok(&meshes[p]) || !decomp_parts_ok(&meshes[p], &decomps[p]))
                return fail(MSDD_ERR_INVALID_ARG, "invalid mesh or decomposition of problem " + std::to_string(p));
            msdd_coeff none{0, nullptr};
            const msdd::Geom g = msdd::make_geom(meshes[p], none);
            const std::vector<msdd::ProbBox> boxes = msdd::make_fine_boxes(g, decomps[p]);
            for (int i = 0; i < (int)boxes.size(); ++i) {
                long long w[3] = {1, 1, 1}, n = 1;
                for (int d = 0; d < meshes[p].dim; ++d) {
                    w[d] = boxes[i].nhi[d] - boxes[i].nlo[d] + 1;
                    n *= w[d];
                }
                // lexicographic half-bandwidth of the Q1 stencil on the Neumann box
                const long long b = meshes[p].dim == 3 ? w[0] * w[1] + w[0] + 1 : w[0] + 1;
                all.push_back({(double)n * (double)(b + 1), p, i});
            }
        }
        std::stable_sort(all.begin(), all.end(), [](const Item& a, const Item& b) { return a.c > b.c; });
        if (count) *count = (long long)all.size();
        // greedy list scheduling in this order: each item to the least loaded
        // worker (lowest index among equals)
        std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>,
                            std::greater<std::pair<double, int>>>
            heap;
        for (int w = 0; w < nworkers; ++w) heap.push({0.0, w});
        double total = 0.0, cmax = 0.0, mk = 0.0;
        for (const Item& it : all) {
            std::pair<double, int> t = heap.top();
            heap.pop();
            t.first += it.c;
            mk = std::max(mk, t.first);
            heap.push(t);
            total += it.c;
            cmax = std::max(cmax, it.c);
        }
        if (makespan) *makespan = mk;
        if (lower_bound) *lower_bound = std::max(total / nworkers, cmax);
        if (items || cost) {
            if (cap < (long long)all.size()) return fail(MSDD_ERR_INVALID_ARG, "buffers smaller than the item count");
            for (size_t k = 0; k < all.size(); ++k) {
                if (items) {
                    items[2 * k] = all[k].p;
                    items[2 * k + 1] = all[k].s;
                }
                if (cost) cost[k] = all[k].c;
            }
        }
        return MSDD_OK;
    });
}

msdd_status msdd_fine_layout(const msdd_mesh* mesh, const msdd_decomp* decomp, int* out, int cap, int* count) {
    return guarded([&]() -> msdd_status {
        if (!mesh_ok(mesh) || !decomp_parts_ok(mesh, decomp)) return fail(MSDD_ERR_INVALID_ARG, "invalid mesh or decomposition");
        msdd::Geom g;
        std::vector<msdd::ProbBox> boxes = warm_boxes(mesh, decomp, g);
        const int P = (int)boxes.size();
        if (count) *count = P;
        if (!out) return MSDD_OK;
        if (cap < 4 * P) return fail(MSDD_ERR_INVALID_ARG, "layout buffer smaller than 4 * subdomains");
        long long off = 0;
        for (int i = 0; i < P; ++i) {
            int nx[3];
            for (int d = 0; d < 3; ++d) nx[d] = d < mesh->dim ? boxes[i].nhi[d] - boxes[i].nlo[d] + 1 : 1;
            if (off > 0x7fffffffLL) return fail(MSDD_ERR_INVALID_ARG, "more than 2^31 rows");
            out[4 * i] = nx[0]; out[4 * i + 1] = nx[1]; out[4 * i + 2] = nx[2]; out[4 * i + 3] = (int)off;
            off += (long long)nx[0] * nx[1] * nx[2];
        }
        return MSDD_OK;
    });
}

msdd_status msdd_nn_patches(const msdd_mesh* mesh, const msdd_coeff* coeff, const msdd_decomp* decomp, float* X,
                            void* stream) {
    return guarded([&]() -> msdd_status {
        if (!mesh_ok(mesh) || !decomp_parts_ok(mesh, decomp) || !X || !coeff || !coeff->data)
            return fail(MSDD_ERR_INVALID_ARG, "invalid arguments");
        if (mesh->dim != 2 || coeff->kind != 0)
            return fail(MSDD_ERR_UNSUPPORTED, "the warm-start network takes 2D scalar coefficients");
        msdd::Geom g;
        std::vector<msdd::ProbBox> boxes = warm_boxes(mesh, decomp, g);
        g.coeff_kind = 0;
        g.coeff = coeff->data;
        cudaStream_t st = (cudaStream_t)stream;
        msdd::DevBuf<msdd::ProbBox> d_boxes;
        d_boxes.upload(boxes, st);
        msdd::nn_patches(g, d_boxes.p, (int)boxes.size(), X, st);
        MSDD_CUDA(cudaStreamSynchronize(st));
        return MSDD_OK;
    });
}

size_t msdd_nn_workspace_bytes(int batch) {
    return batch < 1 ? 0 : msdd::nn_workspace_floats(batch) * sizeof(float);
}

msdd_status msdd_nn_forward(const float* params, int batch, const float* X, float* out, void* work, void* stream) {
    return guarded([&]() -> msdd_status {
        if (!params || batch < 1 || !X || !out || !work) return fail(MSDD_ERR_INVALID_ARG, "invalid arguments");
        msdd::nn_forward(params, batch, X, out, (float*)work, (cudaStream_t)stream);
        return MSDD_OK;
    });
}

msdd_status msdd_nn_loss_grad(const float* params, int batch, const float* X, const float* T, const int* m,
                              double* loss, float* grad, void* work, void* stream) {
    return guarded([&]() -> msdd_status {
        if (!params || batch < 1 || !X || !T || !m || !loss || !grad || !work)
            return fail(MSDD_ERR_INVALID_ARG, "invalid arguments");
        msdd::nn_loss_grad(params, batch, X, T, m, loss, grad, (float*)work, (cudaStream_t)stream);
        return MSDD_OK;
    });
}

msdd_status msdd_nn_adam(float* params, const float* grad, float* m1, float* m2, int t, float lr, void* stream) {
    return guarded([&]() -> msdd_status {
        if (!params || !grad || !m1 || !m2 || t < 1 || !(lr > 0.f)) return fail(MSDD_ERR_INVALID_ARG, "invalid arguments");
        msdd::nn_adam(params, grad, m1, m2, t, lr, (cudaStream_t)stream);
        return MSDD_OK;
    });
}

msdd_status msdd_nn_start_vectors(const msdd_mesh* mesh, const msdd_decomp* decomp, const float* Y, double* out,
                                  void* stream) {
    return guarded([&]() -> msdd_status {
        if (!mesh_ok(mesh) || !decomp_parts_ok(mesh, decomp) || !Y || !out)
            return fail(MSDD_ERR_INVALID_ARG, "invalid arguments");
        if (mesh->dim != 2) return fail(MSDD_ERR_UNSUPPORTED, "the warm-start network is 2D");
        msdd::Geom g;
        std::vector<msdd::ProbBox> boxes = warm_boxes(mesh, decomp, g);
        std::vector<long long> off(boxes.size());
        long long o = 0;
        for (size_t i = 0; i < boxes.size(); ++i) {
            off[i] = o;
            o += (long long)(boxes[i].nhi[0] - boxes[i].nlo[0] + 1) * (boxes[i].nhi[1] - boxes[i].nlo[1] + 1);
        }
        cudaStream_t st = (cudaStream_t)stream;
        msdd::DevBuf<msdd::ProbBox> d_boxes;
        msdd::DevBuf<long long> d_off;
        d_boxes.upload(boxes, st);
        d_off.upload(off, st);
        msdd::nn_start_vectors(d_boxes.p, d_off.p, (int)boxes.size(), 2, Y, out, st);
        MSDD_CUDA(cudaStreamSynchronize(st));
        return MSDD_OK;
    });
}

msdd_status msdd_nn_targets(const msdd_hierarchy* h, float* T, int* m, void* stream) {
    return guarded([&]() -> msdd_status {
        if (!h || !T || !m) return fail(MSDD_ERR_INVALID_ARG, "invalid arguments");
        const msdd::Hierarchy& H = h->h;
        if (H.g.dim != 2) return fail(MSDD_ERR_UNSUPPORTED, "the warm-start network is 2D");
        cudaStream_t st = (cudaStream_t)stream;
        msdd::nn_targets(H.d_fboxes.p, H.fge.K.d_roff.p, H.fge.m.p, H.Pf, H.g.dim, H.fge.X.p, H.fge.ldx, T, m, st);
        MSDD_CUDA(cudaStreamSynchronize(st));
        return MSDD_OK;
    });
}

}  // extern "C"
