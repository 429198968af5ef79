// Host orchestration of the multilevel spectral DD hierarchy (set-up and CG).
#pragma once
#include <string>
#include <vector>

#include "../../include/msdd.h"
#include "coarse.cuh"
#include "eig.cuh"
#include "pcg.cuh"
#include "q1.cuh"
#include "tile_ldlt.cuh"

namespace msdd {

struct MsddError : std::runtime_error {
    msdd_status status;
    MsddError(msdd_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

// CUDA-event timing of kernel families (options.profile); the bytes and flops
// recorded with each launch are algorithmic amounts computed on the host.
struct Prof {
    bool on = false;
    bool solves_only = false;      // level 2: families whose name ends in "_solve"
    bool skipped = false;          // the open interval was not recorded
    struct Fam {
        std::string name;
        int launches = 0;
        double ms = 0, bytes = 0, flops = 0;
    };
    struct Pending {
        int fam;
        cudaEvent_t a, b;
        double bytes, flops;
    };
    std::vector<Fam> fams;
    std::vector<Pending> pend;
    int family(const std::string& name) {
        for (size_t k = 0; k < fams.size(); ++k)
            if (fams[k].name == name) return (int)k;
        fams.push_back(Fam{name});
        return (int)fams.size() - 1;
    }
    void begin(const std::string& name, cudaStream_t s) {
        if (!on) return;
        skipped = solves_only && !(name.size() >= 6 && name.compare(name.size() - 6, 6, "_solve") == 0);
        if (skipped) return;
        Pending p{family(name), timing_event_get(), timing_event_get(), 0, 0};
        MSDD_CUDA(cudaEventRecord(p.a, s));
        pend.push_back(p);
    }
    void end(cudaStream_t s, double bytes, double flops) {
        if (!on || skipped) return;
        Pending& p = pend.back();
        p.bytes = bytes;
        p.flops = flops;
        MSDD_CUDA(cudaEventRecord(p.b, s));
    }
    void collect() {
        for (Pending& p : pend) {
            MSDD_CUDA(cudaEventSynchronize(p.b));
            float ms = 0.f;
            MSDD_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
            Fam& f = fams[p.fam];
            f.launches += 1;
            f.ms += ms;
            f.bytes += p.bytes;
            f.flops += p.flops;
            timing_event_put(p.a);
            timing_event_put(p.b);
        }
        pend.clear();
    }
};

// Geometry of the mesh (coefficient pointer from coeff) and the fine
// subdomain boxes of a decomposition (Section 2.2 box partition with
// overlap); throws MsddError for a subdomain without interior unknowns.
Geom make_geom(const msdd_mesh& mesh, const msdd_coeff& coeff);
std::vector<ProbBox> make_fine_boxes(const Geom& g, const msdd_decomp& dec);

struct Hierarchy {
    Prof prof;
    // ---- problem
    Geom g{};
    msdd_options opt{};
    msdd_spectral spec{};
    msdd_decomp dec{};
    cudaStream_t st = nullptr;
    bool own_stream = false;           // created when the caller passes no stream
    cudaStream_t st2 = nullptr;        // coarse chain of the preconditioner
    cudaStream_t st3 = nullptr;        // set-up side stream: fine Dirichlet factors
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_dir = nullptr;
    cudaEvent_t ev_chunk[2] = {nullptr, nullptr};   // PCG: completion of the last two graph launches
    void* pinned = nullptr;            // 4 KiB pinned host scratch: eigensolver flags, PCG scalars
    int levels = 0, L = 0;
    long long nun = 0;
    msdd_stats stats{};

    // ---- fine level (level L)
    int Pf = 0;
    std::vector<ProbBox> fboxes;
    DevBuf<ProbBox> d_fboxes;
    DevBuf<int> d_count;
    DevBuf<int> d_ecov[3];          // b^2: per axis, fine element boxes holding each element index
    TileBatch fdir;                 // Dirichlet factors A_{L,i}
    GevpBatch fge;                  // GEVP of (Abar_i, B_i), K_i factors
    LocalStencil fst;               // stored stencils of Abar_i and B_i (rows of fge)
    std::vector<int> fm;            // selected counts m_i
    DevBuf<int> d_fm;
    int ldphi = 1;
    std::vector<long long> phioff;
    DevBuf<long long> d_phioff;
    DevBuf<double> Phi;             // chi_i w_{i,k} on the Dirichlet boxes
    std::vector<long long> c1off;   // offset of subdomain i's block in V_{h,L-1}
    DevBuf<long long> d_c1off;
    long long n1 = 0;
    DevBuf<int> cm_first[3], cm_last[3];
    CombineMaps cmaps{};
    DevBuf<double> frhs;            // fine solve buffer
    DevBuf<double> A1;              // dense Galerkin matrix of level L-1 (n1 x n1)

    // ---- middle level (levels == 3, level 1)
    int Pm = 0;
    std::vector<std::vector<int>> members, gens;
    std::vector<int> nown, ngen, c1first;
    std::vector<long long> aoff;
    DevBuf<long long> d_aoff;
    DevBuf<int> d_ngen, d_nown;
    DevBuf<double> Abar_m, K_m;
    TileBatch mdir;
    GevpBatch mge;
    std::vector<int> mm;
    int ldz = 1;
    std::vector<long long> zoff;
    DevBuf<double> Zb;
    std::vector<long long> c0off;
    DevBuf<double> Tm;              // A_1 Z_1
    DevBuf<double> v1, z1t;         // restricted residual / coarse correction on V_{h,1}
    std::vector<long long> moff;
    DevBuf<double> Minv;            // explicit A_{1,i}^{-1}
    DevBuf<GemmItem> d_gemm_y1, d_gemm_r0, d_gemm_z1;
    int gemm_y1_maxm = 0, gemm_r0_maxm = 0, gemm_z1_maxm = 0;

    // ---- coarsest level
    long long n0 = 0;
    TileBatch cdir;
    DevBuf<double> A0, A0inv;       // A_0 and its explicit inverse
    DevBuf<double> r0buf, y0buf;
    DevBuf<GemmItem> d_gemm_y0;

    // ---- CG
    DevBuf<double> x, r, p, q, z, partial;
    DevBuf<double> stencil;         // stored 3^d-point global operator
    DevBuf<double> coeff_own;       // the hierarchy's copy of the element coefficients
    DevBuf<PcgScalars> sc;
    int nblocks = 1;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    long long graph_kernels = 0;

    ~Hierarchy();
    void setup(const msdd_mesh& mesh, const msdd_coeff& coeff);
    // fin_sc: the CG scalars whose beta step the final combine applies (PCG)
    void apply_prec(const double* rr, double* zz, const int* gdone, PcgScalars* fin_sc = nullptr);
    int solve(const double* b, double tol, int maxit, double* xout, double* relres);
    // hybrid form (multiplicative over levels, restricted additive Schwarz on
    // the fine level) and right-preconditioned GMRES with it (Section 5)
    DevBuf<double> hyb_t, hyb_q;
    DevBuf<GemmItem> d_gemm_a1;     // v1 -= A_1 z1 (one n1 x n1 item)
    void apply_hybrid(const double* rr, double* zz, const int* done = nullptr);
    int solve_gmres(const double* b, double tol, int restart, int maxit, double* xout, double* relres);
    size_t device_bytes() const;

   private:
    void build_fine();
    void build_coarse();
    void build_graph();
    void export_prof();
};

}  // namespace msdd
