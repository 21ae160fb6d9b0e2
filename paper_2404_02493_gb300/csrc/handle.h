// Host-side state of one mg_handle (internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "../../include/wave_adr.h"

namespace wadr {

constexpr int MAXB = 2048;          // partial-sum capacity (blocks per segment)
constexpr int MAX_LEVELS = 16;

struct LevelHost {
    int n = 0, pitch = 0;           // nodes per row, row pitch (elements)
    int ny = 0;                     // rows
    double h = 0;
    size_t slot_stride = 0;         // elements
    int nslot = 0;
    void* vec = nullptr;            // slots (cycle precision)
    void* kf = nullptr;             // k (cycle precision)
    void* sig = nullptr;            // sponge term (cycle precision) or null
    void* adr = nullptr;            // ADR quads (cycle precision) or null
    void* mod = nullptr;            // level 2 modulation (cycle precision) or null
    double* k64 = nullptr;          // k in FP64 (setup, outer loop at level 1)
    double* phi64 = nullptr;        // phi in FP64 (setup, adjoint)
    double* sig64 = nullptr;        // sponge term in FP64 or null
    void* inv_helm = nullptr;       // coarsest only: dense inverses in the cycle precision
    void* inv_adr = nullptr;
    double lam_max = 0, alpha = 0;  // Chebyshev interval (levels with Chebyshev)
    double peclet = 0;              // ADR levels: omega h max(|phi_x|, |phi_y|) (condition: <= 1)
    double omega_j = 0;             // Jacobi levels: the damping weight
    int cheb = 0;                   // uses Chebyshev smoothing
    int desc = -1;                  // index in the cycle descriptor table
};

struct InstHost {
    int n = 0, ny = 0, L = 0, bc = 0;   // fine grid: n nodes per row, ny rows
    int la = 0;                     // level of the ADR corrections (0: none)
    int adr_flags = 0;              // ADR_ABC | ADR_DISC options of the ADR coefficients (see adr_coef_at)
    double omega = 0;
    double omega_j = 0;
    std::vector<LevelHost> lv;      // lv[0] = level 1
    // outer FP64 level-1 vectors (slots SU, SG, SD, SX2)
    void* outer_vec = nullptr;
    void* kv = nullptr;             // FGMRES Krylov vectors (cycle precision)
    size_t outer_stride = 0;
    int outer_desc = -1;
    long long off = 0;              // offset of this instance in user arrays (elements)
    // Wave-Ray: the ADR levels of corrections m = 2..M (rv[m-2][l-1], l >= 2):
    // own phase, ADR quads, level-2 modulation, coarsest inverse and
    // descriptor; slots and k shared with lv.  Correction 1 uses lv itself.
    std::vector<std::vector<LevelHost>> rv;
};

struct SegTable {
    Seg* d = nullptr;
    int nseg = 0, nblocks = 0;     // nseg < 0: a single segment, descriptor -nseg - 1
    bool outer = false;            // descriptors of the outer (FP64) table
    long long pts = 0;     // sum of n ny over the segments
    long long mat = 0;     // sum of (n ny)^2 (dense coarsest matrices)
};

// kernel kinds for the event profiler (names in kernel_kind_name)
enum KernelKind : int {
    KK_RESTRICT_JAC0 = 0, KK_RESTRICT_HELM, KK_GS_PRE, KK_PROLONG_JAC, KK_PROLONG_ADD, KK_PROLONG_ADR,
    KK_CHEB, KK_RESDEMOD, KK_GS_GRAM, KK_GS_POST, KK_COARSE, KK_OUTER_RESIDUAL, KK_OUTER_SCALE, KK_OUTER_UPDATE,
    KK_JACOBI, KK_FG_START, KK_FG_PREP, KK_FG_MATVEC, KK_FG_DOTS, KK_FG_ORTH, KK_FG_UPDATE, KK_ADR_TAIL, KK_WAVE_TAIL, KK_COUNT
};
const char* kernel_kind_name(int k);

// halo-tile candidates (index into the gs_*_shape tables) of one ADR launch
struct TileChoice {
    int gram = -1, pre = -1;   // -1: default shape
};

std::string desc_key(const std::vector<int>& descs);
// Blocks per segment of a launch: every segment at least one, the rest of
// the cap given greedily to the segment with the most work units per block.
std::vector<int> share_blocks(const std::vector<long long>& units, int cap);

struct Handle {
    mg_params p{};
    int prec = MG_PREC_FP64;        // cycle precision
    std::vector<InstHost> inst;
    int Lmax = 0;
    // descriptor tables (device) and host copies
    std::vector<LevelDesc> hdesc;   // cycle levels of all instances (Wave-Ray variants after the base levels)
    std::vector<int> base_of;       // descriptor -> the base descriptor of its (instance, level)
    int cur_var = 0;                // Wave-Ray: correction whose ADR descriptors the engine emits
    LevelDesc* ddesc = nullptr;
    std::vector<LevelDesc> houter;  // outer FP64 level-1 descriptors
    LevelDesc* douter = nullptr;
    double* scal = nullptr;         // [ndesc + ninst][S::SIZE]
    double2* part = nullptr;        // [ndesc + ninst][MAXB][MAXDOT]
    unsigned* counter = nullptr;    // [ndesc + ninst][NCOUNTERS]
    void* tmaps = nullptr;          // [ndesc][NMAP] tensor maps of the tile kernels
    unsigned* err = nullptr;        // device error word (bounded waits that expired)
    std::map<std::string, SegTable> segs;
    std::map<std::string, TileChoice> tiles;  // per ADR launch (desc_key), from the autotuner
    std::map<std::string, int*> tail_first;   // per coarse-tail launch: first-level descriptors (device)
    int wave_tail_nmax = 0;                    // wave-cycle levels l >= 4 with n_l <= this run as the shared-memory tail
    int roles[MAX_LEVELS] = {};                // effective role of level l (l >= 2, below an instance's coarsest)
    std::vector<void*> allocs;      // everything cudaMalloc'ed
    size_t alloc_bytes = 0;         // their total size
    long long alloc_limit = 0;      // mg_params.workspace_limit (0: none)
    long long total_elems = 0;      // sum of n ny over instances
    // graphs
    cudaGraphExec_t g_cycle0 = nullptr;     // cycle from u = 0 (level-1 SG -> SD)
    cudaGraphExec_t g_irstep = nullptr;     // scale + cycle + update + residual
    cudaStream_t g_stream = nullptr;
    int launches_cycle = 0;                 // kernels of the last emitted cycle
    int launches_step = 0;                  // kernels of the last emitted outer step
    // event profiler (mg_profile_steps)
    int prof = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> prof_kind;
    std::vector<double> prof_bytes;
    std::vector<long long> prof_pts;        // points of each profiled launch
    bool solve_ready = false;               // mg_solve_begin was called
    // FGMRES
    int fg_j = 0;                           // inner index of the current restart (host copy)
    double* fs = nullptr;                   // [ninst][FS::SIZE]
    double2* fpart = nullptr;               // [ninst][MAXB][NVL]
    double* est = nullptr;                  // [ninst]
    cudaGraphExec_t g_fgiter = nullptr;
    // pinned host scratch for scalars
    double* hpin = nullptr;
    unsigned* herr = nullptr;               // pinned copy of the device error word
    std::string last_error;

    void* alloc(size_t bytes);
    const SegTable& seg(const std::vector<int>& descs, bool outer, int pts_per_block);
    const SegTable& seg_rows(const std::vector<int>& descs, int rows_per_block);
    // one block per tile of tx x ty nodes (of the next level when `coarse`), at most cap per segment
    const SegTable& seg_tiles(const std::vector<int>& descs, int tx, int ty, bool coarse, int cap);
    // outer descriptors: one block per `chunk` values of the padded level-1 array, at most cap per segment
    const SegTable& seg_outer_chunks(const std::vector<int>& descs, int chunk, int cap);
};

// level operations of EngineBase::level_op
enum LevelOp : int {
    OP_APPLY = 0, OP_RESIDUAL, OP_RESTRICT, OP_PROLONG, OP_JACOBI, OP_CHEB, OP_GMRES, OP_ADRV, OP_ADRCORR,
    OP_COARSE
};

// engine interface (one implementation per cycle precision)
struct EngineBase {
    virtual ~EngineBase() {}
    virtual int setup_fields(Handle& H, const mg_instance* in, cudaStream_t st) = 0;
    virtual void cycle(Handle& H, bool uzero, cudaStream_t st) = 0;
    virtual void ir_step(Handle& H, cudaStream_t st) = 0;
    virtual void outer_residual(Handle& H, bool gnorm, cudaStream_t st) = 0;
    virtual void fg_start(Handle& H, cudaStream_t st) = 0;
    virtual void fg_iter(Handle& H, cudaStream_t st) = 0;
    virtual void fg_finish(Handle& H, cudaStream_t st) = 0;
    // level operations (single instance) used by the parity tests
    virtual int level_op(Handle& H, int inst, int level, int what, int a0, int a1, cudaStream_t st) = 0;
    // halo-tile autotuner of the ADR launches (fills Handle::tiles)
    virtual int autotune(Handle& H, cudaStream_t st) = 0;
};

EngineBase* make_engine_f32();
EngineBase* make_engine_f64();

// setup helpers shared by the engines (setup.cu)
// (n nodes per row, ny rows, row pitch `pitch`)
void setup_plane_phase(double* phi64, int n, int ny, int pitch, double h1, int scale, double cx, double cy,
                       cudaStream_t st);
void setup_inject(const double* k_fine, const double* phi_fine, int n1, int ny1, double omega, int bc,
                  double sponge_width, double sponge_power, int level, double* k64, double* phi64, double* sig64, int n,
                  int ny, int pitch, cudaStream_t st);
double setup_lambda_max(const double* k64, const double* sig64, int n, int ny, int pitch, double h, int bc,
                        double shift, double* dscratch, cudaStream_t st);
double setup_adr_scale(const double* k64, const double* phi64, const double* sig64, int n, int ny, int pitch,
                       double h, double omega, int bc, double shift, int adr_flags, double* dscratch,
                       cudaStream_t st);
int setup_check_fields(const double* k, const double* phi, int n, int ny, double* dscratch, long long* bad_k,
                       long long* bad_phi, cudaStream_t st);
double setup_peclet(const double* k64, const double* phi64, const double* sig64, int n, int ny, int pitch, double h,
                    double omega, int bc, double* dscratch, cudaStream_t st);
int setup_coarse_inverse(const double* k64, const double* phi64, const double* sig64, int n, int ny, int pitch,
                         double h, double omega, int bc, double shift, int which, int adr_flags, void* inv, int single,
                         cudaStream_t st);

#define WADR_CHECK(x)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) {                                                        \
            set_error(std::string(#x) + ": " + cudaGetErrorString(e_));                 \
            return MG_ECUDA;                                                            \
        }                                                                               \
    } while (0)

void set_error(const std::string& s);
void prof_begin(Handle& H, cudaStream_t st);
void prof_end(Handle& H, cudaStream_t st, int kind, double bytes, long long pts);

}  // namespace wadr

struct mg_handle {
    wadr::Handle H;
    wadr::EngineBase* eng = nullptr;
};
