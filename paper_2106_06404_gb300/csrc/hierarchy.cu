// Set-up of the multilevel spectral DD hierarchy and the CG solve.
//
// Set-up follows the recursive construction of Section 2.3:
//   fine level L: local Dirichlet matrices (Eq. dirichlet_space) factorised;
//     local GEVPs (Eq. theGEVP with abar of Eq. locala_cg and b^1 of Eq.
//     cg_rhs_blf) by batched subspace iteration; coarse basis
//     phi = e chi w for the selected eigenpairs (Eq. coarse_space_def).
//   level L-1: Galerkin matrix from patch Gram blocks (Section 4.1);
//     with three levels, generating-system Neumann matrices (Section 4.2),
//     regularised factorisation, dense GEVPs, next coarse basis.
//   level 0: one direct factorisation.
#include "hierarchy.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>

namespace msdd {

namespace {

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

void split_axis(int N, int P, std::vector<int>& s, std::vector<int>& e) {
    s.resize(P);
    e.resize(P);
    int base = N / P, rem = N % P, cur = 0;
    for (int p = 0; p < P; ++p) {
        s[p] = cur;
        cur += base + (p < rem ? 1 : 0);
        e[p] = cur;
    }
}

int box_bandwidth(const int lo[3], const int hi[3], int dim) {
    int w0 = hi[0] - lo[0] + 1;
    if (dim == 2) return w0 + 1;
    int w1 = hi[1] - lo[1] + 1;
    return w0 * w1 + w0 + 1;
}

int host_box_size(const int lo[3], const int hi[3], int dim) { return box_size(lo, hi, dim); }

template <typename T>
DevBuf<T> upload_vec(const std::vector<T>& h, cudaStream_t s) {
    DevBuf<T> d;
    d.upload(h, s);
    return d;
}

void check_status(const TileBatch& tb, cudaStream_t s, const char* what) {
    std::vector<int> stv = tb.d_status.download(s);
    for (int i = 0; i < (int)stv.size(); ++i)
        if (stv[i] != 0)
            throw MsddError(MSDD_ERR_NOT_SPD, std::string(what) + ": non-positive pivot in problem " +
                                                  std::to_string(i) + " at row " + std::to_string(stv[i] - 1));
}

int sum_nreg(const TileBatch& tb, cudaStream_t s) {
    std::vector<int> v = tb.d_nreg.download(s);
    int t = 0;
    for (int x : v) t += x;
    return t;
}

// Dense (pseudo-)inverse of every factorised problem of a tile batch:
// out[ooff[i] + r * ld[i] + c] = (K_i^+)[r][c] for r, c < n[i].  The identity
// columns are solved in blocks of 32 columns, one CTA per (problem, block),
// so the whole GPU works on it.
void dense_inverse(const TileBatch& tb, double* out, const std::vector<long long>& ooff, const std::vector<int>& ld,
                   cudaStream_t st) {
    int maxn = 0;
    for (int v : tb.n) maxn = std::max(maxn, v);
    const int lde = tb.max_K * NB;
    DevBuf<double> E((size_t)tb.total_rows * lde);
    tile_identity(tb, E.p, lde, st);
    tile_solve(tb, E.p, lde, maxn, nullptr, st);
    std::vector<CopyItem> ci(tb.P);
    for (int i = 0; i < tb.P; ++i) {
        ci[i].soff = tb.roff[i] * lde;
        ci[i].lds = lde;
        ci[i].doff = ooff[i];
        ci[i].ldd = ld[i];
        ci[i].rows = tb.n[i];
        ci[i].cols = tb.n[i];
    }
    DevBuf<CopyItem> d_ci = upload_vec(ci, st);
    copy_blocks(d_ci.p, tb.P, E.p, out, st);
    MSDD_CUDA(cudaStreamSynchronize(st));
}

// Subspace iteration driver.  apply(v, p0, X, AX, BX, skip, s) applies Abar
// and B to the problems of batch view v (first problem p0 of the whole
// batch), solve(v, p0, ncols, s) applies K^{-1} to v.W, bapply32(v, p0, X, W, s)
// is the FP32 B apply.  `tag` names the kernel families for profiling;
// `apply_bytes`/`apply_flops` are the algorithmic amounts of one operator
// application per problem.
//
// With groups = 2 the problems are split into two halves on two streams
// whose iterations are offset by about one band solve: the latency-bound
// kernels of one half (band solve, Rayleigh-Ritz) then run beside the
// FP64-bound kernels of the other (operators, Gram products, updates).
// Convergence is read back every `batch` = 4 iterations (a host round trip
// per iteration would drain the stream); a group that converged inside a
// batch only launches kernels that skip its (done) problems.
//
// With `fused` (operators cheaper than the p x p update: stored stencils),
// the update forms X = Y C only and apply_rhs(v, p0, s) applies Abar and B
// to the new X, writing the next right-hand side W and the residual partial
// sums; AX and BX are then not kept.
template <class Apply, class Solve, class BApply32, class ApplyRhs>
void run_eig(GevpBatch& g, const EigParams& ep, Apply apply, Solve solve, BApply32 bapply32, ApplyRhs apply_rhs,
             bool fused, int fp32_iters, cudaStream_t st, cudaStream_t st_b, Prof& prof, const std::string& tag,
             double apply_bytes, double apply_flops, int* h_act, const double* start = nullptr,
             int start_cols = 0, const long long* d_start_off = nullptr, int groups = 1) {
    if (g.P == 0) return;
    eig_init(g, ep.seed, st);
    eig_load_start(g, start, start_cols, d_start_off, st);
    const int G = (groups == 2 && g.P >= 2 && st_b) ? 2 : 1;
    const int batch = 4;
    std::vector<GevpBatch> gv;
    std::vector<int> gp0;
    std::vector<cudaStream_t> gs;
    if (G == 1) {
        gv.push_back(g.slice(0, g.P, 0));
        gp0 = {0};
        gs = {st};
    } else {
        const int h = g.P / 2;
        gv.push_back(g.slice(0, h, 0));
        gv.push_back(g.slice(h, g.P - h, 1));
        gp0 = {0, h};
        gs = {st, st_b};
    }
    cudaEvent_t ev_start, ev_off, ev_end;
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_off, cudaEventDisableTiming));
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_end, cudaEventDisableTiming));
    MSDD_CUDA(cudaEventRecord(ev_start, st));
    for (int k = 1; k < G; ++k) MSDD_CUDA(cudaStreamWaitEvent(gs[k], ev_start, 0));
    struct Amounts { int pm = 0; double sb0 = 0, sf0 = 0, solve_b = 0, solve_f = 0, vec_n = 0; };
    std::vector<Amounts> am(G);
    for (int k = 0; k < G; ++k) {
        const GevpBatch& v = gv[k];
        const double fsz = v.K.prec ? 4.0 : 8.0;
        for (int i = 0; i < v.P; ++i) {
            const double n = v.K.n[i], b = v.K.b[i], p = v.p[i];
            am[k].pm = std::max(am[k].pm, v.p[i]);
            // factor band read by both sweeps; right-hand sides read once and
            // solutions written once (FP64)
            am[k].sb0 += 2.0 * n * (b + 1) * fsz + 2.0 * n * p * 8.0;
            am[k].sf0 += 4.0 * n * b * p;
            am[k].vec_n += n * p;
        }
        am[k].solve_b = am[k].sb0;
        am[k].solve_f = am[k].sf0;
    }
    // FP32 start phase: block inverse iteration Y = K~^{-1} B X with Euclidean
    // CholQR, all in FP32 arithmetic; the FP64 phase below starts from its
    // subspace and alone decides convergence.
    for (int it = 0; it < fp32_iters; ++it)
        for (int k = 0; k < G; ++k) {
            GevpBatch& v = gv[k];
            prof.begin(tag + "_fp32_start_other", gs[k]);
            bapply32(v, gp0[k], v.X.p, v.W.p, gs[k]);
            prof.end(gs[k], 0.0, 0.0);
            prof.begin(tag + "_solve", gs[k]);
            solve(v, gp0[k], am[k].pm, gs[k]);
            prof.end(gs[k], am[k].sb0, am[k].sf0);
            if (G == 2 && k == 0 && it == 0) {
                MSDD_CUDA(cudaEventRecord(ev_off, gs[0]));        // the second half starts one solve later
                MSDD_CUDA(cudaStreamWaitEvent(gs[1], ev_off, 0));
            }
            prof.begin(tag + "_fp32_start_other", gs[k]);
            eig_cholqr32(v, gs[k]);
            prof.end(gs[k], 0.0, 0.0);
        }
    std::vector<int> active(G), iter(G, 0);
    for (int k = 0; k < G; ++k) {
        active[k] = gv[k].P;
        apply(gv[k], gp0[k], gv[k].X.p, gv[k].AX.p, gv[k].BX.p, (const int*)nullptr, gs[k]);
    }
    // one iteration of half k on its stream; returns whether it ran a convergence test
    auto iteration = [&](int k, int it, bool offset) -> bool {
        GevpBatch& v = gv[k];
        cudaStream_t s = gs[k];
        const bool first = it == 0;
        const double fr = (double)active[k] / v.P;
        if (!fused || first) eig_form_rhs(v, ep.sigma, first, s);
        prof.begin(tag + "_solve", s);
        solve(v, gp0[k], am[k].pm, s);
        prof.end(s, am[k].solve_b * fr, am[k].solve_f * fr);
        if (offset) {
            MSDD_CUDA(cudaEventRecord(ev_off, s));
            MSDD_CUDA(cudaStreamWaitEvent(gs[1], ev_off, 0));
        }
        if (v.knorm && !first) {
            // test the current Ritz pairs before updating them
            eig_form_y_knorm(v, ep.sigma, s);
            MSDD_CUDA(cudaMemsetAsync(v.n_active.p, 0, sizeof(int), s));
            eig_check_knorm(v, ep, it, s);
        } else {
            eig_form_y(v, ep.sigma, first, s);
        }
        prof.begin(tag + "_apply", s);
        apply(v, gp0[k], v.Y.p, v.AY.p, v.BY.p, (const int*)v.done.p, s);
        prof.end(s, apply_bytes * active[k], apply_flops * active[k]);
        prof.begin(tag + "_gram", s);
        eig_gram(v, s);
        prof.end(s, 3.0 * am[k].vec_n * 8.0 * fr, 2.0 * am[k].vec_n * (am[k].pm + 1) * fr);
        prof.begin(tag + "_rayleigh_ritz", s);
        eig_rayleigh_ritz(v, s);
        prof.end(s, 0.0, 0.0);
        if (fused) {
            prof.begin(tag + "_update", s);
            eig_update_x(v, s);
            prof.end(s, 2.0 * am[k].vec_n * 8.0 * fr, 2.0 * am[k].vec_n * am[k].pm * fr);
            prof.begin(tag + "_apply", s);
            apply_rhs(v, gp0[k], s);
            prof.end(s, (apply_bytes + 8.0 * am[k].vec_n / std::max(1, v.P)) * active[k], apply_flops * active[k]);
        } else {
            prof.begin(tag + "_update", s);
            eig_update(v, s);
            prof.end(s, 6.0 * am[k].vec_n * 8.0 * fr, 6.0 * am[k].vec_n * am[k].pm * fr);
        }
        if (v.knorm) {
            if (first) return false;
        } else {
            MSDD_CUDA(cudaMemsetAsync(v.n_active.p, 0, sizeof(int), s));
            eig_check(v, ep, it, s);
        }
        MSDD_CUDA(cudaMemcpyAsync(&h_act[k], v.n_active.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        return true;
    };
    for (;;) {
        bool any = false;
        std::vector<bool> checked(G, false);
        for (int b = 0; b < batch; ++b)
            for (int k = 0; k < G; ++k) {
                if (active[k] == 0 || iter[k] >= ep.maxit) continue;
                const bool offset = G == 2 && k == 0 && b == 0 && active[1] > 0 && iter[1] < ep.maxit;
                if (iteration(k, iter[k], offset)) checked[k] = true;
                ++iter[k];
                any = true;
            }
        if (!any) break;
        for (int k = 0; k < G; ++k) {
            MSDD_CUDA(cudaStreamSynchronize(gs[k]));
            if (checked[k]) active[k] = h_act[k];
        }
        bool more = false;
        for (int k = 0; k < G; ++k) more = more || (active[k] > 0 && iter[k] < ep.maxit);
        if (!more) break;
    }
    for (int k = 1; k < G; ++k) {
        MSDD_CUDA(cudaEventRecord(ev_end, gs[k]));
        MSDD_CUDA(cudaStreamWaitEvent(st, ev_end, 0));
    }
    MSDD_CUDA(cudaStreamSynchronize(st));
    cudaEventDestroy(ev_start);
    cudaEventDestroy(ev_off);
    cudaEventDestroy(ev_end);
    int left = 0;
    for (int k = 0; k < G; ++k) left += active[k];
    if (g.knorm && left > 0) {
        // eig_maxit reached: the last updated pairs are kept and marked unconverged
        std::vector<int> dn = g.done.download(st);
        for (int& v : dn)
            if (v == 0) v = 2;
        g.done.upload(dn, st);
    }
    prof.collect();
}

}  // namespace

Hierarchy::~Hierarchy() {
    if (graph) cudaGraphExecDestroy(graph);
    if (st2) {
        cudaStreamSynchronize(st2);
        cudaStreamDestroy(st2);
    }
    if (st3) {
        cudaStreamSynchronize(st3);
        cudaStreamDestroy(st3);
    }
    if (ev_dir) cudaEventDestroy(ev_dir);
    for (cudaEvent_t& e : ev_chunk)
        if (e) cudaEventDestroy(e);
    pinned_cache_release(pinned, 4096);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (own_stream && st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
}

Geom make_geom(const msdd_mesh& mesh, const msdd_coeff& coeff) {
    Geom g{};
    g.dim = mesh.dim;
    for (int d = 0; d < 3; ++d) g.n[d] = d < mesh.dim ? mesh.n[d] : 1;
    for (int d = 0; d < 3; ++d) {
        if (d < mesh.dim) {
            g.ulo[d] = (mesh.dirichlet_faces >> (2 * d)) & 1 ? 1 : 0;
            g.uhi[d] = (mesh.dirichlet_faces >> (2 * d + 1)) & 1 ? g.n[d] - 1 : g.n[d];
        } else {
            g.ulo[d] = g.uhi[d] = 0;
        }
        g.ushape[d] = g.uhi[d] - g.ulo[d] + 1;
    }
    g.coeff_kind = coeff.kind;
    g.ncomp = coeff.kind == 0 ? 1 : (mesh.dim == 2 ? 3 : 6);
    g.coeff = coeff.data;
    g.rscale = mesh.dim == 3 ? 1.0 / g.n[0] : 1.0;
    return g;
}

std::vector<ProbBox> make_fine_boxes(const Geom& g, const msdd_decomp& dec) {
    const int dim = g.dim;
    std::vector<int> s[3], e[3];
    for (int d = 0; d < 3; ++d) {
        int P = d < dim ? dec.parts[d] : 1;
        split_axis(g.n[d], P, s[d], e[d]);
    }
    int P0 = dec.parts[0], P1 = dim >= 2 ? dec.parts[1] : 1, P2 = dim == 3 ? dec.parts[2] : 1;
    std::vector<ProbBox> boxes(P0 * P1 * P2);
    for (int pz = 0; pz < P2; ++pz)
        for (int py = 0; py < P1; ++py)
            for (int px = 0; px < P0; ++px) {
                int j = px + P0 * (py + P1 * pz);
                int pi[3] = {px, py, pz};
                ProbBox& b = boxes[j];
                for (int d = 0; d < 3; ++d) {
                    if (d >= dim) {
                        b.elo[d] = 0; b.ehi[d] = 1;
                        b.nlo[d] = b.nhi[d] = b.dlo[d] = b.dhi[d] = 0;
                        continue;
                    }
                    int lo = std::max(0, s[d][pi[d]] - dec.overlap);
                    int hi = std::min(g.n[d], e[d][pi[d]] + dec.overlap);
                    b.elo[d] = lo;
                    b.ehi[d] = hi;
                    b.nlo[d] = std::max(lo, g.ulo[d]);
                    b.nhi[d] = std::min(hi, g.uhi[d]);
                    int dlo = lo == 0 ? 0 : lo + 1;
                    int dhi = hi == g.n[d] ? g.n[d] : hi - 1;
                    b.dlo[d] = std::max(dlo, g.ulo[d]);
                    b.dhi[d] = std::min(dhi, g.uhi[d]);
                }
                if (host_box_size(b.dlo, b.dhi, dim) <= 0 || host_box_size(b.nlo, b.nhi, dim) <= 0)
                    throw MsddError(MSDD_ERR_INVALID_ARG, "subdomain " + std::to_string(j) + " has no interior unknowns");
            }
    return boxes;
}

size_t Hierarchy::device_bytes() const {
    size_t b = 0;
    b += fdir.bytes() + fge.K.bytes() + cdir.bytes() + mdir.bytes() + mge.K.bytes();
    b += (fge.X.n + fge.AX.n + fge.BX.n + fge.Y.n + fge.AY.n + fge.BY.n + fge.W.n) * 8;
    b += (mge.X.n + mge.AX.n + mge.BX.n + mge.Y.n + mge.AY.n + mge.BY.n + mge.W.n) * 8;
    b += (Phi.n + A1.n + Abar_m.n + K_m.n + Zb.n + Tm.n + A0.n + frhs.n + v1.n + r0buf.n) * 8;
    b += (Minv.n + A0inv.n + y0buf.n + z1t.n) * 8;
    b += (x.n + r.n + p.n + q.n + z.n + stencil.n + coeff_own.n) * 8;
    b += (fst.a.n + fst.b.n) * 8 + fst.b32.n * 4;
    return b;
}

void Hierarchy::setup(const msdd_mesh& mesh, const msdd_coeff& coeff) {
    auto t_all = Clock::now();
    if (!st) {
        // graph capture needs a stream other than the legacy default one; a
        // blocking stream keeps the legacy stream's ordering for the caller
        MSDD_CUDA(cudaStreamCreate(&st));
        own_stream = true;
    }
    MSDD_CUDA(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    MSDD_CUDA(cudaStreamCreateWithFlags(&st3, cudaStreamNonBlocking));
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_dir, cudaEventDisableTiming));
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_chunk[0], cudaEventDisableTiming));
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_chunk[1], cudaEventDisableTiming));
    pinned = pinned_cache_alloc(4096);
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    MSDD_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
    levels = dec.levels;
    L = levels - 1;
    prof.on = opt.profile != 0;
    prof.solves_only = opt.profile == 2;
    g = make_geom(mesh, coeff);
    {
        // the caller's coefficient array is read here only: later set-up work
        // and msdd_apply_operator use the hierarchy's own copy
        const long long ne = (long long)g.n[0] * g.n[1] * g.n[2] * g.ncomp;
        coeff_own.alloc((size_t)ne);
        MSDD_CUDA(cudaMemcpyAsync(coeff_own.p, coeff.data, (size_t)ne * sizeof(double), cudaMemcpyDeviceToDevice, st));
        g.coeff = coeff_own.p;
    }
    nun = (long long)g.ushape[0] * g.ushape[1] * g.ushape[2];
    // node coordinates in the combine kernel use 32-bit divisions
    if (nun >= (1LL << 31)) throw MsddError(MSDD_ERR_UNSUPPORTED, "more than 2^31 unknowns");
    upload_reference(g);

    memset(&stats, 0, sizeof(stats));
    stats.n = nun;
    stats.levels = levels;
    stats.precision = opt.precision;

    build_fine();
    build_coarse();
    // the fine Dirichlet factors ran on st3 beside the eigensolves
    MSDD_CUDA(cudaStreamWaitEvent(st, ev_dir, 0));
    check_status(fdir, st, "fine Dirichlet factorisation");

    // CG buffers and the stored global stencil
    x.alloc(nun); r.alloc(nun); p.alloc(nun); q.alloc(nun); z.alloc(nun);
    stencil.alloc((size_t)nun * (g.dim == 3 ? 27 : 9));
    global_stencil(g, stencil.p, st);
    nblocks = dot_blocks(nun);
    partial.alloc(nblocks);
    sc.alloc(1);
    MSDD_CUDA(cudaMemsetAsync(sc.p, 0, sizeof(PcgScalars), st));
    MSDD_CUDA(cudaStreamSynchronize(st));
    tile_check_waits();
    stats.setup_ms = ms_since(t_all);
    stats.device_bytes = device_bytes();
    export_prof();
}

void Hierarchy::export_prof() {
    stats.nprof = (int)std::min<size_t>(prof.fams.size(), MSDD_MAX_PROF);
    for (int k = 0; k < stats.nprof; ++k) {
        const Prof::Fam& f = prof.fams[k];
        memset(stats.prof[k].name, 0, sizeof(stats.prof[k].name));
        strncpy(stats.prof[k].name, f.name.c_str(), sizeof(stats.prof[k].name) - 1);
        stats.prof[k].launches = f.launches;
        stats.prof[k].ms = f.ms;
        stats.prof[k].bytes = f.bytes;
        stats.prof[k].flops = f.flops;
    }
}

void Hierarchy::build_fine() {
    auto t0 = Clock::now();
    const int dim = g.dim;
    int P0 = dec.parts[0], P1 = dim >= 2 ? dec.parts[1] : 1, P2 = dim == 3 ? dec.parts[2] : 1;
    Pf = P0 * P1 * P2;
    fboxes = make_fine_boxes(g, dec);
    d_fboxes = upload_vec(fboxes, st);
    // right-hand side of the fine GEVPs (Section 3.4); b^2 needs to know which
    // elements lie in more than one fine box (per axis: boxes are products)
    g.blf = spec.blf == 0 ? 1 : spec.blf;
    if (g.blf == 2) {
        const int stride[3] = {1, P0, P0 * P1}, np[3] = {P0, P1, P2};
        for (int d = 0; d < dim; ++d) {
            std::vector<int> cov(g.n[d], 0);
            for (int q = 0; q < np[d]; ++q) {
                const ProbBox& b = fboxes[q * stride[d]];
                for (int x = b.elo[d]; x < b.ehi[d]; ++x) ++cov[x];
            }
            d_ecov[d] = upload_vec(cov, st);
            g.ecov[d] = d_ecov[d].p;
        }
    }
    // combine maps: per axis and node coordinate, the blocks whose Dirichlet range holds it
    cmaps.parts[0] = P0; cmaps.parts[1] = P1; cmaps.parts[2] = P2;
    for (int d = 0; d < 3; ++d) {
        int nn = g.n[d] + 1;
        std::vector<int> fi(nn, 0), la(nn, -1);
        if (d < dim) {
            int Pd = dec.parts[d];
            for (int x = 0; x < nn; ++x) {
                fi[x] = -1;
                la[x] = -2;
                for (int p = 0; p < Pd; ++p) {
                    int idx[3] = {0, 0, 0};
                    idx[d] = p;
                    int j = idx[0] + P0 * (idx[1] + P1 * idx[2]);
                    if (x >= fboxes[j].dlo[d] && x <= fboxes[j].dhi[d]) {
                        if (fi[x] < 0) fi[x] = p;
                        la[x] = p;
                    }
                }
                if (x >= g.ulo[d] && x <= g.uhi[d] && fi[x] < 0)
                    throw MsddError(MSDD_ERR_INVALID_ARG, "node not interior to any subdomain: overlap must be >= 1");
                if (fi[x] < 0) { fi[x] = 0; la[x] = -1; }
            }
        } else {
            fi.assign(nn, 0);
            la.assign(nn, 0);
        }
        cm_first[d] = upload_vec(fi, st);
        cm_last[d] = upload_vec(la, st);
        cmaps.first[d] = cm_first[d].p;
        cmaps.last[d] = cm_last[d].p;
    }
    d_count.alloc(nun);
    pou_count(g, d_fboxes.p, Pf, d_count.p, st);
    MSDD_CUDA(cudaStreamSynchronize(st));
    stats.phase_ms[0] = ms_since(t0);

    // ---- Dirichlet factors: only the preconditioner needs them, so they are
    // assembled and factored on the side stream st3, beside the Neumann
    // factors and the fine eigensolves (ev_dir marks completion; their status
    // is checked at the end of the set-up)
    t0 = Clock::now();
    std::vector<int> nD(Pf), bD(Pf), nN(Pf), bN(Pf);
    for (int j = 0; j < Pf; ++j) {
        nD[j] = host_box_size(fboxes[j].dlo, fboxes[j].dhi, dim);
        bD[j] = box_bandwidth(fboxes[j].dlo, fboxes[j].dhi, dim);
        nN[j] = host_box_size(fboxes[j].nlo, fboxes[j].nhi, dim);
        bN[j] = box_bandwidth(fboxes[j].nlo, fboxes[j].nhi, dim);
    }
    const int prec = opt.precision ? 1 : 0;
    fdir.layout(nD, bD, prec, st);
    MSDD_CUDA(cudaStreamSynchronize(st));            // layout tables uploaded
    tile_zero(fdir, st3);
    assemble_local_tiles(g, d_fboxes.p, d_count.p, fdir, 0, 0.0, st3);
    {
        double fb = 0, ff = 0, sz = prec ? 4.0 : 8.0;
        for (int j = 0; j < Pf; ++j) {
            fb += 2.0 * nD[j] * (bD[j] + 1.0) * sz;
            ff += (double)nD[j] * bD[j] * bD[j];
        }
        prof.begin("fine_factor", st3);
        tile_factor(fdir, 0.0, st3);
        prof.end(st3, fb, ff);
    }
    MSDD_CUDA(cudaEventRecord(ev_dir, st3));
    frhs.alloc(fdir.total_rows);
    frhs.zero(st);
    MSDD_CUDA(cudaStreamSynchronize(st));
    stats.phase_ms[1] = ms_since(t0);

    // ---- shifted Neumann factors K = Abar + sigma B
    t0 = Clock::now();
    fge.K.layout(nN, bN, prec, st);
    tile_zero(fge.K, st);
    assemble_local_tiles(g, d_fboxes.p, d_count.p, fge.K, 1, opt.sigma, st);
    {
        double fb = 0, ff = 0, sz = prec ? 4.0 : 8.0;
        for (int j = 0; j < Pf; ++j) {
            fb += 2.0 * nN[j] * (bN[j] + 1.0) * sz;
            ff += (double)nN[j] * bN[j] * bN[j];
        }
        prof.begin("fine_factor", st);
        tile_factor(fge.K, 0.0, st);
        prof.end(st, fb, ff);
        prof.collect();
    }
    check_status(fge.K, st, "fine shifted Neumann factorisation");
    MSDD_CUDA(cudaStreamSynchronize(st));
    stats.phase_ms[2] = ms_since(t0);

    // ---- fine GEVPs
    t0 = Clock::now();
    const int block_p = opt.block_p > 0 ? opt.block_p : std::min(spec.nev_max + 4, PMAX);
    fge.ldx = PMAX;
    fge.p.resize(Pf);
    for (int j = 0; j < Pf; ++j) fge.p[j] = std::min(block_p, nN[j]);
    fge.alloc(st);
    EigParams ep;
    ep.sigma = opt.sigma;
    ep.tol = opt.eig_tol;
    ep.eta = spec.eta;
    ep.nev_max = spec.nev_max;
    ep.maxit = opt.eig_maxit;
    ep.seed = opt.seed;
    build_local_stencil(g, d_fboxes.p, d_count.p, fge.K, fst, st);
    DevBuf<long long> d_woff;              // row offsets of the caller's start vectors
    if (opt.warm_start) {
        std::vector<long long> woff(Pf);
        long long o = 0;
        for (int j = 0; j < Pf; ++j) { woff[j] = o; o += nN[j]; }
        d_woff = upload_vec(woff, st);
    }
    const ProbBox* bx = d_fboxes.p;
    const LocalStencil* ls = &fst;
    double nav = 0;
    for (int j = 0; j < Pf; ++j) nav += nN[j];
    nav /= Pf;
    run_eig(fge, ep,
            [=](GevpBatch& v, int p0, const double* X, double* AX, double* BX, const int* skip, cudaStream_t s) {
                apply_local(*ls, bx + p0, dim, v.K, X, AX, BX, v.ldx, block_p, skip, s);
            },
            [=](GevpBatch& v, int, int pmax, cudaStream_t s) { tile_solve(v.K, v.W.p, v.ldx, pmax, v.done.p, s); },
            [=](GevpBatch& v, int p0, const double* X, double* W, cudaStream_t s) {
                apply_local_b32(*ls, bx + p0, dim, v.K, X, W, v.ldx, block_p, s);
            },
            [=](GevpBatch& v, int p0, cudaStream_t s) {
                apply_local_rhs(*ls, bx + p0, dim, v.K, v.X.p, v.W.p, v.ldx, v.d_p.p, v.theta.p, ep.sigma,
                                v.partial.p, v.nblk_max, v.done.p, s);
            },
            true, opt.precision == 1 ? opt.fp32_start_iters : 0,
            st, st2, prof, "fine_gevp", nav * (3.0 * block_p * 8.0 + 8.0), nav * block_p * 2.0 * 2.0 * (dim == 3 ? 27 : 9),
            static_cast<int*>(pinned), opt.warm_start, opt.warm_start ? opt.warm_cols : 0, d_woff.p, Pf >= 64 ? 2 : 1);
    fm = fge.m.download(st);
    {
        std::vector<int> it = fge.iters.download(st), dn = fge.done.download(st);
        int mx = 0, mn = 1 << 30, unc = 0, mmin = 1 << 30, mmax = 0;
        for (int j = 0; j < Pf; ++j) {
            mx = std::max(mx, it[j]);
            mn = std::min(mn, it[j]);
            unc += dn[j] == 2 ? 1 : 0;
            stats.eig_at_floor[L] += dn[j] == 3 ? 1 : 0;
            mmin = std::min(mmin, fm[j]);
            mmax = std::max(mmax, fm[j]);
        }
        stats.eig_iters_max[L] = mx;
        stats.eig_iters_min[L] = mn;
        for (int j = 0; j < Pf; ++j) stats.eig_iters_total[L] += it[j];
        stats.eig_unconverged[L] = unc;
        stats.m_min[L] = mmin;
        stats.m_max[L] = mmax;
        stats.subdomains[L] = Pf;
    }
    d_fm = upload_vec(fm, st);
    ldphi = std::max(1, spec.nev_max);
    phioff.resize(Pf);
    long long tot = 0;
    for (int j = 0; j < Pf; ++j) {
        phioff[j] = tot;
        tot += (long long)nD[j] * ldphi;
    }
    Phi.alloc(tot);
    d_phioff = upload_vec(phioff, st);
    make_coarse_basis(g, d_fboxes.p, d_count.p, fge.K, fge.X.p, fge.ldx, d_fm.p, Phi.p, d_phioff.p, ldphi, Pf, st);
    MSDD_CUDA(cudaStreamSynchronize(st));
    stats.phase_ms[3] = ms_since(t0);
}

void Hierarchy::build_coarse() {
    auto t0 = Clock::now();
    const int dim = g.dim;
    const int P0 = cmaps.parts[0], P1 = cmaps.parts[1], P2 = cmaps.parts[2];
    // ---- level L-1 ordering of the fine subdomains (group-major with 3 levels)
    std::vector<int> order;
    if (levels == 3) {
        int G[3] = {1, 1, 1};
        int Pp[3] = {P0, P1, P2};
        std::vector<int> gs[3], ge[3];
        for (int d = 0; d < 3; ++d) {
            int gd = d < dim ? std::max(1, Pp[d] / std::max(1, dec.group[d])) : 1;
            G[d] = gd;
            split_axis(Pp[d], gd, gs[d], ge[d]);
        }
        Pm = G[0] * G[1] * G[2];
        members.assign(Pm, {});
        for (int qz = 0; qz < G[2]; ++qz)
            for (int qy = 0; qy < G[1]; ++qy)
                for (int qx = 0; qx < G[0]; ++qx) {
                    int i = qx + G[0] * (qy + G[1] * qz);
                    for (int pz = gs[2][qz]; pz < ge[2][qz]; ++pz)
                        for (int py = gs[1][qy]; py < ge[1][qy]; ++py)
                            for (int px = gs[0][qx]; px < ge[0][qx]; ++px)
                                members[i].push_back(px + P0 * (py + P1 * pz));
                    std::sort(members[i].begin(), members[i].end());
                    for (int j : members[i]) order.push_back(j);
                }
    } else {
        for (int j = 0; j < Pf; ++j) order.push_back(j);
    }
    c1off.assign(Pf, 0);
    n1 = 0;
    for (int j : order) {
        c1off[j] = n1;
        n1 += fm[j];
    }
    stats.level_dim[L] = nun;
    stats.level_dim[L - 1] = n1;
    d_c1off = upload_vec(c1off, st);
    if (n1 == 0) throw MsddError(MSDD_ERR_UNSUPPORTED, "empty coarse space (no eigenvalue below eta)");

    // ---- patches: per axis, runs of elements with equal block-membership intervals
    struct AxisPatch { int e0, e1, plo, phi; };
    std::vector<AxisPatch> ap[3];
    for (int d = 0; d < 3; ++d) {
        if (d >= dim) { ap[d].push_back({0, 1, 0, 0}); continue; }
        int Pd = dec.parts[d];
        int prev_lo = -1, prev_hi = -1, start = 0;
        for (int x = 0; x <= g.n[d]; ++x) {
            int lo = -1, hi = -1;
            if (x < g.n[d]) {
                for (int p = 0; p < Pd; ++p) {
                    int idx[3] = {0, 0, 0};
                    idx[d] = p;
                    const ProbBox& b = fboxes[idx[0] + P0 * (idx[1] + P1 * idx[2])];
                    if (x >= b.elo[d] && x < b.ehi[d]) {
                        if (lo < 0) lo = p;
                        hi = p;
                    }
                }
            }
            if (x == g.n[d] || lo != prev_lo || hi != prev_hi) {
                if (x > 0 && prev_lo >= 0) ap[d].push_back({start, x, prev_lo, prev_hi});
                start = x;
                prev_lo = lo;
                prev_hi = hi;
            }
        }
    }
    struct Patch { int elo[3], ehi[3]; std::vector<int> mem; };
    std::vector<Patch> patches;
    for (auto& az : ap[2])
        for (auto& ay : ap[1])
            for (auto& ax : ap[0]) {
                Patch pt;
                const AxisPatch* a3[3] = {&ax, &ay, &az};
                for (int d = 0; d < 3; ++d) { pt.elo[d] = a3[d]->e0; pt.ehi[d] = a3[d]->e1; }
                for (int pz = az.plo; pz <= az.phi; ++pz)
                    for (int py = ay.plo; py <= ay.phi; ++py)
                        for (int px = ax.plo; px <= ax.phi; ++px) pt.mem.push_back(px + P0 * (py + P1 * pz));
                patches.push_back(std::move(pt));
            }
    std::vector<GramItem> gitems;
    std::vector<long long> gpatch;       // patch index of each item
    long long gtot = 0;
    for (size_t k = 0; k < patches.size(); ++k) {
        for (int j : patches[k].mem)
            for (int jj : patches[k].mem) {
                if (fm[j] == 0 || fm[jj] == 0) continue;
                GramItem it;
                for (int d = 0; d < 3; ++d) { it.elo[d] = patches[k].elo[d]; it.ehi[d] = patches[k].ehi[d]; }
                it.j = j;
                it.jj = jj;
                it.goff = gtot;
                gtot += (long long)fm[j] * fm[jj];
                gitems.push_back(it);
                gpatch.push_back((long long)k);
            }
    }
    DevBuf<GramItem> d_gitems = upload_vec(gitems, st);
    DevBuf<double> G(std::max<long long>(gtot, 1));
    patch_gram(g, d_fboxes.p, Phi.p, d_phioff.p, ldphi, d_fm.p, d_gitems.p, (int)gitems.size(), G.p, st);

    // ---- Galerkin matrix of level L-1: block (j, jj) = sum over patches holding both
    std::map<std::pair<int, int>, std::vector<long long>> pairc;
    for (size_t k = 0; k < gitems.size(); ++k) pairc[{gitems[k].j, gitems[k].jj}].push_back(gitems[k].goff);
    {
        std::vector<SumItem> si;
        std::vector<long long> contrib;
        for (auto& kv : pairc) {
            int j = kv.first.first, jj = kv.first.second;
            SumItem it;
            it.doff = c1off[j] * n1 + c1off[jj];
            it.ld = (int)n1;
            it.rows = fm[j];
            it.cols = fm[jj];
            it.cbeg = (int)contrib.size();
            for (long long c : kv.second) contrib.push_back(c);
            it.cend = (int)contrib.size();
            si.push_back(it);
        }
        A1.alloc(n1 * n1);
        A1.zero(st);
        DevBuf<SumItem> d_si = upload_vec(si, st);
        DevBuf<long long> d_contrib = upload_vec(contrib, st);
        block_sum(d_si.p, (int)si.size(), d_contrib.p, G.p, A1.p, st);
        MSDD_CUDA(cudaStreamSynchronize(st));
    }
    stats.phase_ms[4] = ms_since(t0);

    if (levels == 2) {
        t0 = Clock::now();
        n0 = n1;
        cdir.layout({(int)n0}, {(int)n0 - 1}, 0, st);
        std::vector<long long> so = {0};
        std::vector<int> ld = {(int)n1};
        DevBuf<long long> d_so = upload_vec(so, st);
        DevBuf<int> d_ld = upload_vec(ld, st);
        tile_from_dense(cdir, A1.p, d_so.p, d_ld.p, st);
        tile_factor(cdir, 0.0, st);
        check_status(cdir, st, "coarse factorisation");
        // A_0^{-1} explicitly: the coarse solve in CG is one GEMV over many CTAs
        A0inv.alloc(n0 * n0);
        dense_inverse(cdir, A0inv.p, {0}, {(int)n0}, st);
        r0buf.alloc(n0);
        r0buf.zero(st);
        y0buf.alloc(n0);
        {
            GemmItem a;
            a.aoff = 0; a.lda = (int)n0;
            a.boff = 0; a.ldb = 1;
            a.coff = 0; a.ldc = 1;
            a.m = (int)n0; a.n = 1; a.k = (int)n0;
            d_gemm_y0 = upload_vec(std::vector<GemmItem>{a}, st);
        }
        stats.level_dim[0] = n0;
        stats.subdomains[0] = 1;
        MSDD_CUDA(cudaStreamSynchronize(st));
        stats.phase_ms[6] = ms_since(t0);
        return;
    }

    // ---- three levels: middle level 1 on the groups
    t0 = Clock::now();
    nown.assign(Pm, 0);
    c1first.assign(Pm, 0);
    for (int i = 0; i < Pm; ++i) {
        c1first[i] = (int)c1off[members[i][0]];
        for (int j : members[i]) nown[i] += fm[j];
    }
    // Dirichlet matrices: own x own blocks of A_1 (contiguous in group-major order)
    {
        std::vector<int> bw(Pm);
        std::vector<long long> so(Pm);
        std::vector<int> ld(Pm, (int)n1);
        for (int i = 0; i < Pm; ++i) {
            bw[i] = std::max(0, nown[i] - 1);
            so[i] = (long long)c1first[i] * n1 + c1first[i];
            if (nown[i] == 0) throw MsddError(MSDD_ERR_UNSUPPORTED, "level-1 subdomain without coarse functions");
        }
        mdir.layout(nown, bw, 0, st);
        DevBuf<long long> d_so = upload_vec(so, st);
        DevBuf<int> d_ld = upload_vec(ld, st);
        tile_from_dense(mdir, A1.p, d_so.p, d_ld.p, st);
        tile_factor(mdir, 0.0, st);
        check_status(mdir, st, "level-1 Dirichlet factorisation");
        // A_{1,i}^{-1} explicitly: level-1 solves in CG are batched GEMVs
        moff.assign(Pm, 0);
        long long mt = 0;
        for (int i = 0; i < Pm; ++i) {
            moff[i] = mt;
            mt += (long long)nown[i] * nown[i];
        }
        Minv.alloc(mt);
        dense_inverse(mdir, Minv.p, moff, nown, st);
    }
    // generating systems: own children, then neighbours meeting T_{1,i}
    gens.assign(Pm, {});
    ngen.assign(Pm, 0);
    aoff.assign(Pm, 0);
    std::vector<std::vector<int>> genoff(Pm);
    std::vector<std::vector<char>> isown(Pm, std::vector<char>(Pf, 0));
    long long atot = 0;
    for (int i = 0; i < Pm; ++i) {
        int tlo[3], thi[3];
        for (int d = 0; d < 3; ++d) { tlo[d] = 1 << 30; thi[d] = -1; }
        for (int j : members[i]) {
            isown[i][j] = 1;
            for (int d = 0; d < 3; ++d) {
                tlo[d] = std::min(tlo[d], fboxes[j].elo[d]);
                thi[d] = std::max(thi[d], fboxes[j].ehi[d]);
            }
            gens[i].push_back(j);
        }
        for (int j = 0; j < Pf; ++j) {
            if (isown[i][j] || fm[j] == 0) continue;
            bool meet = true;
            for (int d = 0; d < dim; ++d)
                if (fboxes[j].ehi[d] <= tlo[d] || fboxes[j].elo[d] >= thi[d]) meet = false;
            if (meet) gens[i].push_back(j);
        }
        genoff[i].assign(Pf, -1);
        int off = 0;
        for (int j : gens[i]) {
            genoff[i][j] = off;
            off += fm[j];
        }
        ngen[i] = off;
        aoff[i] = atot;
        atot += (long long)off * off;
    }
    Abar_m.alloc(atot);
    Abar_m.zero(st);
    K_m.alloc(atot);
    {
        std::vector<SumItem> si;
        std::vector<long long> contrib;
        for (int i = 0; i < Pm; ++i) {
            std::map<std::pair<int, int>, std::vector<long long>> pc;
            for (size_t k = 0; k < gitems.size(); ++k) {
                int j = gitems[k].j, jj = gitems[k].jj;
                if (genoff[i][j] < 0 || genoff[i][jj] < 0) continue;
                bool touches = false;
                for (int mbr : patches[gpatch[k]].mem)
                    if (isown[i][mbr]) { touches = true; break; }
                if (!touches) continue;
                pc[{j, jj}].push_back(gitems[k].goff);
            }
            for (auto& kv : pc) {
                int j = kv.first.first, jj = kv.first.second;
                SumItem it;
                it.doff = aoff[i] + (long long)genoff[i][j] * ngen[i] + genoff[i][jj];
                it.ld = ngen[i];
                it.rows = fm[j];
                it.cols = fm[jj];
                it.cbeg = (int)contrib.size();
                for (long long c : kv.second) contrib.push_back(c);
                it.cend = (int)contrib.size();
                si.push_back(it);
            }
        }
        DevBuf<SumItem> d_si = upload_vec(si, st);
        DevBuf<long long> d_contrib = upload_vec(contrib, st);
        block_sum(d_si.p, (int)si.size(), d_contrib.p, G.p, Abar_m.p, st);
    }
    d_aoff = upload_vec(aoff, st);
    d_ngen = upload_vec(ngen, st);
    d_nown = upload_vec(nown, st);
    int ngen_max = *std::max_element(ngen.begin(), ngen.end());
    dense_shift(Abar_m.p, K_m.p, d_aoff.p, d_ngen.p, d_nown.p, opt.sigma, Pm, ngen_max, st);
    {
        std::vector<int> bw(Pm);
        for (int i = 0; i < Pm; ++i) bw[i] = std::max(0, ngen[i] - 1);
        mge.K.layout(ngen, bw, 0, st);
    }
    // null-pivot threshold of the generating systems: negative = automatic
    // (1e-10 in 2D, 1e-6 in 3D, whose generating systems carry more
    // near-dependent neighbour generators; a 2D level whose eigensolves do
    // not converge is factored and solved again with 1e-6, below)
    const bool reg_auto = opt.reg_tol < 0.0;
    double reg_tol = reg_auto ? (g.dim == 3 ? 1e-6 : 1e-10) : opt.reg_tol;
    auto factor_K = [&](double rt) {
        tile_from_dense(mge.K, K_m.p, d_aoff.p, d_ngen.p, st);
        tile_factor(mge.K, rt, st);
        stats.null_pivots[1] = sum_nreg(mge.K, st);
        // K^+ explicitly (overwrites K_m): every later solve is a batched GEMM
        dense_inverse(mge.K, K_m.p, aoff, ngen, st);
    };
    factor_K(reg_tol);
    stats.phase_ms[4] += ms_since(t0);
    t0 = Clock::now();
    int block_p = opt.block_p > 0 ? opt.block_p : std::min(spec.nev_max + 8, PMAX);
    mge.ldx = PMAX;
    mge.knorm = true;
    mge.p.resize(Pm);
    for (int i = 0; i < Pm; ++i) mge.p[i] = std::min(block_p, nown[i]);
    mge.alloc(st);
    EigParams ep;
    ep.sigma = opt.sigma;
    ep.tol = opt.eig_tol;
    ep.eta = spec.eta;
    ep.nev_max = spec.nev_max;
    ep.maxit = opt.eig_maxit;
    ep.seed = opt.seed + 7919;
    const double* Ab = Abar_m.p;
    const long long* dao = d_aoff.p;
    const int* dng = d_ngen.p;
    const int* dno = d_nown.p;
    std::vector<GemmItem> kitems(Pm);
    int pmax_m = 0;
    for (int i = 0; i < Pm; ++i) {
        GemmItem& it = kitems[i];
        it.aoff = aoff[i];
        it.lda = ngen[i];
        it.boff = mge.K.roff[i] * mge.ldx;
        it.ldb = mge.ldx;
        it.coff = mge.K.roff[i] * mge.ldx;
        it.ldc = mge.ldx;
        it.m = ngen[i];
        it.n = mge.p[i];
        it.k = ngen[i];
        pmax_m = std::max(pmax_m, mge.p[i]);
    }
    DevBuf<GemmItem> d_kitems = upload_vec(kitems, st);
    DevBuf<double> Wt(mge.W.n);
    std::vector<long long> mrow(Pm + 1);            // first W element of each problem, and the end
    for (int i = 0; i < Pm; ++i) mrow[i] = mge.K.roff[i] * mge.ldx;
    mrow[Pm] = (long long)mge.K.total_rows * mge.ldx;
    const GemmItem* dki = d_kitems.p;
    const double* Kinv = K_m.p;
    double* Wtp = Wt.p;
    auto eig_pass = [&]() {
        stats.eig_at_floor[1] = 0;
        stats.eig_iters_total[1] = 0;
        run_eig(mge, ep,
                [=](GevpBatch& v, int p0, const double* X, double* AX, double* BX, const int* skip, cudaStream_t s) {
                    apply_dense_pencil(Ab, dao + p0, dng + p0, dno + p0, v.K, X, AX, BX, v.ldx, block_p, skip, v.P,
                                       ngen_max, s);
                },
                [=](GevpBatch& v, int p0, int, cudaStream_t s) {
                    gemm_batched(dki + p0, v.P, 0, 0, 1.0, Kinv, v.W.p, 0.0, Wtp, ngen_max, pmax_m, s, nullptr,
                                 v.done.p);
                    const long long e0 = mrow[p0], e1 = mrow[p0 + v.P];
                    MSDD_CUDA(cudaMemcpyAsync(v.W.p + e0, Wtp + e0, (e1 - e0) * sizeof(double),
                                              cudaMemcpyDeviceToDevice, s));
                },
                [=](GevpBatch&, int, const double*, double*, cudaStream_t) {},
                [=](GevpBatch&, int, cudaStream_t) {}, false, 0,
                st, nullptr, prof, "coarse_gevp", (double)ngen_max * ngen_max * 8.0, 2.0 * ngen_max * ngen_max * block_p,
                static_cast<int*>(pinned));
        mm = mge.m.download(st);
        {
            std::vector<int> it = mge.iters.download(st), dn = mge.done.download(st);
            int mx = 0, mn = 1 << 30, unc = 0, mmin = 1 << 30, mmax = 0;
            for (int i = 0; i < Pm; ++i) {
                mx = std::max(mx, it[i]);
                mn = std::min(mn, it[i]);
                unc += dn[i] == 2 ? 1 : 0;
                stats.eig_at_floor[1] += dn[i] == 3 ? 1 : 0;
                mmin = std::min(mmin, mm[i]);
                mmax = std::max(mmax, mm[i]);
            }
            stats.eig_iters_max[1] = mx;
            stats.eig_iters_min[1] = mn;
            for (int i = 0; i < Pm; ++i) stats.eig_iters_total[1] += it[i];
            stats.eig_unconverged[1] = unc;
            stats.m_min[1] = mmin;
            stats.m_max[1] = mmax;
            stats.subdomains[1] = Pm;
        }
    };
    eig_pass();
    // automatic options: problems that did not converge are solved again (all
    // of the level) with the larger null-pivot threshold and the widest block
    // (near-dependent generators; clusters of tiny eigenvalues that a block of
    // nev + 8 separates slowly from the rest of the spectrum)
    const bool block_auto = opt.block_p == 0;
    if (stats.eig_unconverged[1] > 0 && ((reg_auto && reg_tol < 1e-6) || (block_auto && block_p < PMAX))) {
        if (reg_auto && reg_tol < 1e-6) {
            reg_tol = 1e-6;
            dense_shift(Abar_m.p, K_m.p, d_aoff.p, d_ngen.p, d_nown.p, opt.sigma, Pm, ngen_max, st);
            factor_K(reg_tol);
        }
        if (block_auto) {
            block_p = PMAX;
            pmax_m = 0;
            for (int i = 0; i < Pm; ++i) {
                mge.p[i] = std::min(block_p, nown[i]);
                pmax_m = std::max(pmax_m, mge.p[i]);
                kitems[i].n = mge.p[i];
            }
            d_kitems = upload_vec(kitems, st);
            dki = d_kitems.p;
            mge.alloc(st);
        }
        eig_pass();
    }
    stats.phase_ms[5] = ms_since(t0);

    // ---- Z_1 blocks (own generators' coefficients) and A_0 = Z_1^T A_1 Z_1
    t0 = Clock::now();
    ldz = std::max(1, spec.nev_max);
    zoff.assign(Pm, 0);
    c0off.assign(Pm, 0);
    long long ztot = 0;
    n0 = 0;
    std::vector<CopyItem> ci;
    for (int i = 0; i < Pm; ++i) {
        zoff[i] = ztot;
        ztot += (long long)nown[i] * ldz;
        c0off[i] = n0;
        n0 += mm[i];
        CopyItem c;
        c.soff = mge.K.roff[i] * mge.ldx;
        c.lds = mge.ldx;
        c.doff = zoff[i];
        c.ldd = ldz;
        c.rows = nown[i];
        c.cols = mm[i];
        ci.push_back(c);
    }
    if (n0 == 0) throw MsddError(MSDD_ERR_UNSUPPORTED, "empty coarsest space (no level-1 eigenvalue below eta)");
    Zb.alloc(ztot);
    Zb.zero(st);
    {
        DevBuf<CopyItem> d_ci = upload_vec(ci, st);
        copy_blocks(d_ci.p, (int)ci.size(), mge.X.p, Zb.p, st);
        MSDD_CUDA(cudaStreamSynchronize(st));
    }
    Tm.alloc(n1 * n0);
    A0.alloc(n0 * n0);
    {
        std::vector<GemmItem> it1, it2;
        int maxn = 0, maxm = 0;
        for (int i = 0; i < Pm; ++i) {
            GemmItem a;
            a.aoff = c1first[i]; a.lda = (int)n1;
            a.boff = zoff[i]; a.ldb = ldz;
            a.coff = c0off[i]; a.ldc = (int)n0;
            a.m = (int)n1; a.n = mm[i]; a.k = nown[i];
            it1.push_back(a);
            maxn = std::max(maxn, mm[i]);
            GemmItem b;
            b.aoff = zoff[i]; b.lda = ldz;
            b.boff = (long long)c1first[i] * n0; b.ldb = (int)n0;
            b.coff = c0off[i] * n0; b.ldc = (int)n0;
            b.m = mm[i]; b.n = (int)n0; b.k = nown[i];
            it2.push_back(b);
            maxm = std::max(maxm, mm[i]);
        }
        DevBuf<GemmItem> d1 = upload_vec(it1, st), d2 = upload_vec(it2, st);
        gemm_batched(d1.p, Pm, 0, 0, 1.0, A1.p, Zb.p, 0.0, Tm.p, (int)n1, maxn, st);
        gemm_batched(d2.p, Pm, 1, 0, 1.0, Zb.p, Tm.p, 0.0, A0.p, maxm, (int)n0, st);
        MSDD_CUDA(cudaStreamSynchronize(st));
    }
    cdir.layout({(int)n0}, {(int)n0 - 1}, 0, st);
    {
        std::vector<long long> so = {0};
        std::vector<int> ld = {(int)n0};
        DevBuf<long long> d_so = upload_vec(so, st);
        DevBuf<int> d_ld = upload_vec(ld, st);
        tile_from_dense(cdir, A0.p, d_so.p, d_ld.p, st);
        tile_factor(cdir, 0.0, st);
        check_status(cdir, st, "coarsest factorisation");
        A0inv.alloc(n0 * n0);
        dense_inverse(cdir, A0inv.p, {0}, {(int)n0}, st);
    }
    r0buf.alloc(n0);
    r0buf.zero(st);
    y0buf.alloc(n0);
    v1.alloc(n1);
    z1t.alloc(n1);
    {
        std::vector<GemmItem> gy1, g0, g1;
        gemm_y1_maxm = gemm_r0_maxm = gemm_z1_maxm = 0;
        for (int i = 0; i < Pm; ++i) {
            GemmItem y;   // z1t_i = A_{1,i}^{-1} v1_i
            y.aoff = moff[i]; y.lda = nown[i];
            y.boff = c1first[i]; y.ldb = 1;
            y.coff = c1first[i]; y.ldc = 1;
            y.m = nown[i]; y.n = 1; y.k = nown[i];
            gy1.push_back(y);
            gemm_y1_maxm = std::max(gemm_y1_maxm, nown[i]);
            GemmItem a;   // r0_i = Zb_i^T v1_i
            a.aoff = zoff[i]; a.lda = ldz;
            a.boff = c1first[i]; a.ldb = 1;
            a.coff = c0off[i]; a.ldc = 1;
            a.m = mm[i]; a.n = 1; a.k = nown[i];
            g0.push_back(a);
            gemm_r0_maxm = std::max(gemm_r0_maxm, mm[i]);
            GemmItem b;   // z1t_i += Zb_i y0_i
            b.aoff = zoff[i]; b.lda = ldz;
            b.boff = c0off[i]; b.ldb = 1;
            b.coff = c1first[i]; b.ldc = 1;
            b.m = nown[i]; b.n = 1; b.k = mm[i];
            g1.push_back(b);
            gemm_z1_maxm = std::max(gemm_z1_maxm, nown[i]);
        }
        d_gemm_y1 = upload_vec(gy1, st);
        d_gemm_r0 = upload_vec(g0, st);
        d_gemm_z1 = upload_vec(g1, st);
        GemmItem a;   // y0 = A_0^{-1} r0
        a.aoff = 0; a.lda = (int)n0;
        a.boff = 0; a.ldb = 1;
        a.coff = 0; a.ldc = 1;
        a.m = (int)n0; a.n = 1; a.k = (int)n0;
        d_gemm_y0 = upload_vec(std::vector<GemmItem>{a}, st);
    }
    stats.level_dim[0] = n0;
    stats.subdomains[0] = 1;
    MSDD_CUDA(cudaStreamSynchronize(st));
    stats.phase_ms[6] = ms_since(t0);
}

void Hierarchy::apply_prec(const double* rr, double* zz, const int* gdone, PcgScalars* fin_sc) {
    double* r1 = levels == 2 ? r0buf.p : v1.p;
    fine_gather_restrict(g, d_fboxes.p, fdir.d_roff.p, fdir.d_K.p, rr, frhs.p, Phi.p, d_phioff.p, ldphi, d_fm.p,
                         d_c1off.p, r1, Pf, gdone, st);
    // the coarse chain runs on a second stream, concurrently with the fine solves
    MSDD_CUDA(cudaEventRecord(ev_fork, st));
    MSDD_CUDA(cudaStreamWaitEvent(st2, ev_fork, 0));
    const double* zc;
    if (levels == 2) {
        gemv_batched(d_gemm_y0.p, 1, 0, 1.0, A0inv.p, r0buf.p, 0.0, y0buf.p, (int)n0, st2, gdone);
        zc = y0buf.p;
    } else {
        gemv_batched(d_gemm_y1.p, Pm, 0, 1.0, Minv.p, v1.p, 0.0, z1t.p, gemm_y1_maxm, st2, gdone);
        gemv_batched(d_gemm_r0.p, Pm, 1, 1.0, Zb.p, v1.p, 0.0, r0buf.p, gemm_r0_maxm, st2, gdone);
        gemv_batched(d_gemm_y0.p, 1, 0, 1.0, A0inv.p, r0buf.p, 0.0, y0buf.p, (int)n0, st2, gdone);
        gemv_batched(d_gemm_z1.p, Pm, 0, 1.0, Zb.p, y0buf.p, 1.0, z1t.p, gemm_z1_maxm, st2, gdone);
        zc = z1t.p;
    }
    MSDD_CUDA(cudaEventRecord(ev_join, st2));
    tile_solve(fdir, frhs.p, 1, 1, nullptr, st, gdone);
    MSDD_CUDA(cudaStreamWaitEvent(st, ev_join, 0));
    fine_combine(g, cmaps, d_fboxes.p, fdir.d_roff.p, frhs.p, Phi.p, d_phioff.p, ldphi, d_fm.p, d_c1off.p, zc, zz,
                 rr, partial.p, nblocks, gdone, st, fin_sc, fin_sc ? PCG_FIN_BETA : PCG_FIN_NONE);
}

void Hierarchy::build_graph() {
    const int chunk = 8;
    cudaGraph_t gr;
    const long long c0 = kernel_launch_counter();
    MSDD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int* gd = &sc.p->done;
    for (int k = 0; k < chunk; ++k) {
        // the finishing steps (alpha, the r.r test, beta) run in the last
        // block of the kernel that produced their partial sums
        spmv_stencil_dot(g, stencil.p, p.p, q.p, partial.p, nblocks, gd, st, sc.p, PCG_FIN_ALPHA);
        pcg_axpy(sc.p, x.p, r.p, p.p, q.p, nun, partial.p, nblocks, st, true);
        apply_prec(r.p, z.p, gd, sc.p);
        pcg_update_p(sc.p, z.p, p.p, nun, st);
    }
    MSDD_CUDA(cudaStreamEndCapture(st, &gr));
    MSDD_CUDA(cudaGraphInstantiate(&graph, gr, 0));
    cudaGraphDestroy(gr);
    graph_iters = chunk;
    graph_kernels = kernel_launch_counter() - c0;   // captured, not launched
    kernel_launch_counter() = c0;
}

int Hierarchy::solve(const double* b, double tol, int maxit, double* xout, double* relres) {
    auto t0 = Clock::now();
    if (!graph) {
        build_graph();
        stats.phase_ms[7] = ms_since(t0);
    }
    pcg_start(b, x.p, r.p, nun, partial.p, nblocks, st);
    pcg_fin_bb(sc.p, partial.p, nblocks, tol, maxit, st);
    apply_prec(r.p, z.p, &sc.p->done);
    pcg_fin_rho0(sc.p, partial.p, nblocks, z.p, p.p, nun, st);
    PcgScalars hs{};
    // algorithmic amounts of one CG iteration: ~10 FP64 vector passes, the
    // fine Dirichlet factors read twice, the coarse basis read twice
    double it_bytes = 10.0 * 8.0 * nun, it_flops = 0.0;
    {
        double sz = fdir.prec ? 4.0 : 8.0;
        for (int j = 0; j < Pf; ++j) {
            it_bytes += 2.0 * fdir.n[j] * (fdir.b[j] + 1.0) * sz + 2.0 * fdir.n[j] * fm[j] * 8.0;
            it_flops += 4.0 * fdir.n[j] * fdir.b[j] + 4.0 * fdir.n[j] * fm[j];
        }
        it_flops += 2.0 * (g.dim == 3 ? 27 : 9) * nun + 10.0 * nun;
    }
    // graph chunks are launched one ahead of the convergence check, so the
    // GPU never waits for the host; a chunk launched after convergence finds
    // the done flag set and its kernels return at once
    PcgScalars* hsc = reinterpret_cast<PcgScalars*>(static_cast<char*>(pinned) + 1024);
    auto launch_chunk = [&](int slot) {
        prof.begin("pcg_iterations", st);
        MSDD_CUDA(cudaGraphLaunch(graph, st));
        kernel_launch_counter() += graph_kernels;
        prof.end(st, 0.0, 0.0);
        MSDD_CUDA(cudaMemcpyAsync(&hsc[slot], sc.p, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        MSDD_CUDA(cudaEventRecord(ev_chunk[slot], st));
    };
    launch_chunk(0);
    launch_chunk(1);
    int prev_iters = 0;
    for (int k = 0;; ++k) {
        const int slot = k & 1;
        MSDD_CUDA(cudaEventSynchronize(ev_chunk[slot]));
        hs = hsc[slot];
        if (prof.on && prof.pend.size() >= 2) {
            // the profiled interval of chunk k is the (k+1)-th pending entry
            Prof::Pending& pe = prof.pend[prof.pend.size() - 2];
            const int done_it = hs.iters - prev_iters;
            pe.bytes = it_bytes * done_it;
            pe.flops = it_flops * done_it;
            prev_iters = hs.iters;
        }
        if (hs.done) break;
        launch_chunk(slot);
    }
    MSDD_CUDA(cudaStreamSynchronize(st));
    prof.collect();
    MSDD_CUDA(cudaMemcpyAsync(xout, x.p, nun * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MSDD_CUDA(cudaStreamSynchronize(st));
    tile_check_waits();
    double rel = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    if (relres) *relres = rel;
    stats.pcg_iterations = hs.iters;
    stats.pcg_rel_residual = rel;
    stats.solve_ms = ms_since(t0);
    export_prof();
    if (hs.done == 3) throw MsddError(MSDD_ERR_NOT_SPD, "CG breakdown: p^T A p <= 0");
    if (hs.done == 2) return -hs.iters;
    return hs.iters;
}

// z = B_h r: the fine level as restricted additive Schwarz (local solutions
// weighted by chi = 1/N(x)), then each coarser level in turn on the current
// residual, z <- z + B_l (r - A z), down to the coarsest (Section 2.1, Eq.
// subspace_iteration applied level by level; the order is a reading).  With
// three levels the coarsest level's residual is formed on level 1: its space
// Phi Z_1 lies in level 1's space Phi, so Z_1^T Phi^T (r - A (z + Phi z1)) =
// Z_1^T (v1 - A_1 z1) with the Galerkin matrix A_1 = Phi^T A Phi and
// v1 = Phi^T (r - A z); both coarse corrections are then prolonged together.
// All on the main stream; every kernel returns at once when `done` is set.
void Hierarchy::apply_hybrid(const double* rr, double* zz, const int* done) {
    double* r1 = levels == 2 ? r0buf.p : v1.p;
    if ((long long)hyb_t.n < nun) {
        hyb_t.alloc(nun);
        hyb_q.alloc(nun);
    }
    if (levels == 3 && !d_gemm_a1.p) {
        GemmItem a;
        a.aoff = 0; a.lda = (int)n1;
        a.boff = 0; a.ldb = 1;
        a.coff = 0; a.ldc = 1;
        a.m = (int)n1; a.n = 1; a.k = (int)n1;
        d_gemm_a1 = upload_vec(std::vector<GemmItem>{a}, st);
    }
    fine_gather_restrict(g, d_fboxes.p, fdir.d_roff.p, fdir.d_K.p, rr, frhs.p, Phi.p, d_phioff.p, ldphi, d_fm.p,
                         d_c1off.p, r1, Pf, done, st);
    tile_solve(fdir, frhs.p, 1, 1, nullptr, st, done);
    fine_combine_mode(g, cmaps, d_fboxes.p, fdir.d_roff.p, frhs.p, Phi.p, d_phioff.p, ldphi, d_fm.p, d_c1off.p, r1,
                      zz, rr, nullptr, nblocks, done, COMB_Y | COMB_RAS, st);
    spmv_stencil_dot(g, stencil.p, zz, hyb_q.p, partial.p, nblocks, done, st);
    vec_sub(rr, hyb_q.p, hyb_t.p, nun, st, done);                           // t = r - A z
    fine_gather_restrict(g, d_fboxes.p, fdir.d_roff.p, fdir.d_K.p, hyb_t.p, frhs.p, Phi.p, d_phioff.p, ldphi, d_fm.p,
                         d_c1off.p, r1, Pf, done, st);                      // r1 = Phi^T t
    const double* zc;
    if (levels == 2) {
        gemv_batched(d_gemm_y0.p, 1, 0, 1.0, A0inv.p, r0buf.p, 0.0, y0buf.p, (int)n0, st, done);
        zc = y0buf.p;
    } else {
        gemv_batched(d_gemm_y1.p, Pm, 0, 1.0, Minv.p, v1.p, 0.0, z1t.p, gemm_y1_maxm, st, done);      // z1
        gemv_batched(d_gemm_a1.p, 1, 0, -1.0, A1.p, z1t.p, 1.0, v1.p, (int)n1, st, done);          // v1 -= A_1 z1
        gemv_batched(d_gemm_r0.p, Pm, 1, 1.0, Zb.p, v1.p, 0.0, r0buf.p, gemm_r0_maxm, st, done);
        gemv_batched(d_gemm_y0.p, 1, 0, 1.0, A0inv.p, r0buf.p, 0.0, y0buf.p, (int)n0, st, done);
        gemv_batched(d_gemm_z1.p, Pm, 0, 1.0, Zb.p, y0buf.p, 1.0, z1t.p, gemm_z1_maxm, st, done);    // z1 += Z_1 y0
        zc = z1t.p;
    }
    fine_combine_mode(g, cmaps, d_fboxes.p, fdir.d_roff.p, frhs.p, Phi.p, d_phioff.p, ldphi, d_fm.p, d_c1off.p, zc,
                      zz, rr, nullptr, nblocks, done, COMB_COARSE | COMB_ACC, st);
}

// Flexible GMRES(restart) (Saad) with the hybrid preconditioner: x0 = 0,
// z_k = B_h v_k kept beside the Arnoldi basis and the cycle's update x += Z y,
// so that the residual estimate stays the true residual when the local
// solves run in FP32 (B_h then is no fixed linear map).  Arnoldi with
// classical Gram-Schmidt applied twice; the coefficients, the Hessenberg
// matrix, the Givens rotations and the stop test stay on the device, so the
// host enqueues the steps in chunks and reads the device state one chunk
// behind (kernels return at once after the stop).  The run stops when the
// Arnoldi residual estimate falls below tol ||b|| (the rule of Section 5 on
// the solver's own residual, as the recursive residual stops CG) or the true
// residual at the end of a cycle does; a cycle that reaches the restart
// length restarts from the true residual.  Returns the step count (negative
// at maxit) and the true residual.
int Hierarchy::solve_gmres(const double* b, double tol, int restart, int maxit, double* xout, double* relres) {
    const long long n = nun;
    const int m = restart, nbd = 64, CH = 4;
    DevBuf<double> V((size_t)(m + 1) * n), Z((size_t)m * n), w(n), t(n), x(n), cdev(m + 1),
        part((size_t)(m + 1) * nbd), Hd((size_t)(m + 1) * m), rot((size_t)3 * m + 2);
    DevBuf<GmresState> gst(1);
    double *cs = rot.p, *sn = rot.p + m, *gvd = rot.p + 2 * m, *hinv = rot.p + 3 * m + 1;
    const int* done = &gst.p->done;
    struct Pinned {
        GmresState* p;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        Pinned() : p(static_cast<GmresState*>(pinned_cache_alloc(2 * sizeof(GmresState)))) {}
        ~Pinned() {
            for (auto e : ev)
                if (e) cudaEventDestroy(e);
            pinned_cache_release(p, 2 * sizeof(GmresState));
        }
    } pin;
    for (auto& e : pin.ev) MSDD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

    std::vector<double> hpart(nbd), tmp;
    auto norm = [&](const double* v) {
        vec_mdot(v, 1, v, n, part.p, nbd, st);
        MSDD_CUDA(cudaMemcpyAsync(hpart.data(), part.p, nbd * sizeof(double), cudaMemcpyDeviceToHost, st));
        MSDD_CUDA(cudaStreamSynchronize(st));
        double ss = 0.0;
        for (int q = 0; q < nbd; ++q) ss += hpart[q];
        return std::sqrt(ss);
    };
    auto step = [&](int k) {
        double* zk = Z.p + (size_t)k * n;
        apply_hybrid(V.p + (size_t)k * n, zk, done);                               // z_k = B_h v_k
        spmv_stencil_dot(g, stencil.p, zk, w.p, partial.p, nblocks, done, st);     // w = A z_k
        for (int pass = 0; pass < 2; ++pass) {
            vec_mdot(V.p, k + 1, w.p, n, part.p, nbd, st, done);
            gm_gs_coef(part.p, nbd, k + 1, Hd.p, m, k, cdev.p, pass > 0, gst.p, st);
            vec_comb(w.p, V.p, cdev.p, k + 1, n, -1.0, false, st, done);
        }
        vec_mdot(w.p, 1, w.p, n, part.p, nbd, st, done);
        gm_fin(part.p, nbd, Hd.p, m, k, cs, sn, gvd, hinv, gst.p, st);
        vec_scale_dev(w.p, V.p + (size_t)(k + 1) * n, hinv, n, done, st);
    };

    x.zero(st);
    const double bn = norm(b);
    int it = 0;
    double rel = 0.0;
    bool conv = bn == 0.0;
    if (bn > 0.0) {
        MSDD_CUDA(cudaMemcpyAsync(t.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));   // r = b
        std::vector<double> H, gv(m + 1);
        for (;;) {
            const double beta = norm(t.p);
            vec_scale_to(t.p, V.p, 1.0 / beta, n, st);
            GmresState s0{0, it, maxit, 0, tol * bn};
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            MSDD_CUDA(cudaMemcpyAsync(gst.p, &s0, sizeof(s0), cudaMemcpyHostToDevice, st));
            MSDD_CUDA(cudaMemcpyAsync(gvd, gv.data(), (m + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
            MSDD_CUDA(cudaMemsetAsync(Hd.p, 0, (size_t)(m + 1) * m * sizeof(double), st));
            MSDD_CUDA(cudaStreamSynchronize(st));   // pageable sources above
            int k = 0, slot = 0;
            bool prev = false;
            while (k < m) {
                for (const int kend = std::min(m, k + CH); k < kend; ++k) step(k);
                MSDD_CUDA(cudaMemcpyAsync(pin.p + slot, gst.p, sizeof(GmresState), cudaMemcpyDeviceToHost, st));
                MSDD_CUDA(cudaEventRecord(pin.ev[slot], st));
                slot ^= 1;
                if (prev) {   // the state after the chunk before this one
                    MSDD_CUDA(cudaEventSynchronize(pin.ev[slot]));
                    if (pin.p[slot].done) break;
                }
                prev = true;
            }
            GmresState sf;
            MSDD_CUDA(cudaMemcpyAsync(&sf, gst.p, sizeof(sf), cudaMemcpyDeviceToHost, st));
            MSDD_CUDA(cudaStreamSynchronize(st));
            const int kk = sf.kk;
            it = sf.it;
            H.resize((size_t)kk * m);
            MSDD_CUDA(cudaMemcpyAsync(H.data(), Hd.p, (size_t)kk * m * sizeof(double), cudaMemcpyDeviceToHost, st));
            MSDD_CUDA(cudaMemcpyAsync(gv.data(), gvd, (kk + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
            MSDD_CUDA(cudaStreamSynchronize(st));
            std::vector<double> y(kk);
            for (int i = kk - 1; i >= 0; --i) {
                double v = gv[i];
                for (int j = i + 1; j < kk; ++j) v -= H[(size_t)i * m + j] * y[j];
                y[i] = v / H[(size_t)i * m + i];
            }
            MSDD_CUDA(cudaMemcpyAsync(cdev.p, y.data(), kk * sizeof(double), cudaMemcpyHostToDevice, st));
            vec_comb(x.p, Z.p, cdev.p, kk, n, 1.0, false, st);                 // x += Z y
            spmv_stencil_dot(g, stencil.p, x.p, w.p, partial.p, nblocks, nullptr, st);
            vec_sub(b, w.p, t.p, n, st);                                        // r = b - A x
            rel = norm(t.p) / bn;
            conv = sf.done == 1 || rel < tol;
            if (conv || it >= maxit) break;
        }
    }
    MSDD_CUDA(cudaMemcpyAsync(xout, x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MSDD_CUDA(cudaStreamSynchronize(st));
    tile_check_waits();
    if (relres) *relres = rel;
    return conv ? it : -it;
}

}  // namespace msdd
