// Host-side structures of a graph handle and the host functions shared
// between the library's translation units.
#pragma once

#include <vector>

#include "fj_sort.cuh"

namespace fj {

// Row blocks: rows [blk_row[b], blk_row[b+1]) form block b.  A block either
// holds at most kBlockRows rows whose nonzeros fit in 2*kBlockNnz (staged in
// shared memory), or is a single long row.
constexpr int kBlockNnz = 1024;
constexpr int kBlockRows = 512;
// Warp tiles of the sweep: rows whose nonzeros fit in 2 * kWarpNnz (sixteen
// per lane), at most kWarpRows rows (two per lane); a longer row is cut into
// chunks of kWarpChunk nonzeros (sixteen per lane: one batch of loads).
// Column and weight arrays carry kNnzPad spare entries, so that the sweep's
// 256-nonzero chunks (16-byte loads of eight entries per lane) and 16-byte
// asynchronous copies of a tile rounded out to 4-element granules stay inside
// the allocation.  The spare entries are never used as values.
constexpr int kNnzPad = 256;
constexpr int kWarpNnz = 256;
constexpr int kWarpRows = 64;
constexpr int kWarpChunk = 512;
// Tilings of a CSR: metric blocks, warp tiles.
enum TileKind { kTileBlock = 0, kTileWarp = 1 };

// One CSR resident on the device plus the per-row arrays the push needs.
struct DevCSR {
    int64_t n = 0, nnz = 0;
    int64_t *row_ptr = nullptr;
    int32_t *col = nullptr;
    float *w = nullptr;        // nullptr = unit weights
    mutable int wexp = INT32_MIN;  // max|w| < 2^wexp, set by the first certificate (weights are fixed)
    double *deg64 = nullptr;   // weighted out-degree d_u (FP64)
    float *inv32 = nullptr;    // float(1 / (1 + d_u))
    double *inv64 = nullptr;   // 1 / (1 + d_u)
    int32_t *indeg = nullptr;  // number of in-neighbours (residual updates per push)
    int32_t *graph_of = nullptr;  // ragged: graph id of each row (nullptr for one graph)
    int32_t *blk_row = nullptr;   // nblocks + 1 entries (block tiles)
    int64_t nblocks = 0;
    int32_t *wblk_row = nullptr;  // nwblocks + 1 entries (warp tiles)
    int64_t nwblocks = 0;
    std::vector<int64_t> seg_blk;  // host: block ranges of forced segments (classes / graphs)
};

// Multicolour order: classes of the symmetrised graph, nodes renumbered so
// that every class is a contiguous range of rows.
struct Colouring {
    bool built = false;
    int palette = -1;           // palette size the colouring was built with (0 = unbounded)
    int ncolours = 0;
    double *din_p = nullptr;    // permuted order: weight to neighbours of the same colour
    int32_t *colour = nullptr;  // by original id
    int32_t *perm = nullptr;    // new id -> original id
    int32_t *iperm = nullptr;   // original id -> new id
    // host: the non-hub rows of class c are [class_row[c], class_row[c+1]) and its
    // hub rows [hub_row[c], hub_row[c+1]); the nhub hubs (nodes of largest
    // in-degree) come first, ordered by class, so hub_row[ncolours] = nhub =
    // class_row[0].  Without hubs every class is the one range of class_row.
    std::vector<int64_t> class_row;
    std::vector<int64_t> hub_row;
    int64_t nhub = 0;
    DevCSR pcsr;                     // permuted CSR, blocks never straddle a class
    // directed graphs, built on first use: in-neighbour lists in the permuted
    // order (row i lists the new ids of the nodes that listen to perm[i])
    int64_t *tptr = nullptr;
    int32_t *tcol = nullptr;
    float *tw = nullptr;
};

// Work items of a sweep, in the order of the sweep (colour order for the
// multicolour schedule).  An item is a row block (slot < 0) or one chunk of a
// long row (slot = the long row's index; its chunks sum into part[] and the
// last one to finish applies the row's update).  lo is the first row of the
// item's colour class: a column below lo belongs to an earlier class.
struct Item {
    int32_t r0, r1;
    int32_t lo;
    int32_t slot;
    int32_t hlo;   // first hub row of the item's class (hub ids below it are in earlier classes)
    int32_t nhub;  // number of hubs (ids below it are hubs); 0 without a hub prefix
    int64_t k0, k1;
};
// Largest hub prefix of the colour order: the fused sweep's hot table holds
// this many FP32 increments in shared memory.
constexpr int kHubMax = 49152;
constexpr int kChunkNnz = 2048;

struct ItemPlan {
    bool built = false;
    Item *items = nullptr;       // device
    int64_t nitems = 0;
    int64_t nslots = 0;          // long rows
    int32_t *slot_first = nullptr;  // device: first chunk index of each long row into part[]
    int32_t *slot_nchunk = nullptr; // device
    double *part = nullptr;         // device: one partial sum per chunk (two words: hi, lo)
    int32_t *cnt = nullptr;         // device: chunks finished per long row
    int64_t nparts = 0;
    std::vector<int64_t> class_item;  // host: items of class c are [class_item[c], class_item[c+1])
};

// Chunk plan of a CSR for the single-vector sweep: the nonzeros cut into
// 256-element chunks (chunk C holds nonzeros 256C .. 256C + 255).
constexpr int kChunkE = 256;
struct ChunkPlan {
    bool built = false;
    int64_t nch = 0;              // chunks
    uint32_t *starts = nullptr;   // 8 (nch + 1) words: bit b of word i set when nonzero 32i + b is the first
                                  // of a non-empty row; one more start at nonzero nnz closes the last row
    int32_t *endbase = nullptr;   // nch entries: non-empty rows that end before chunk C
    int32_t *rank = nullptr;      // n entries: non-empty rows before row x (row x's slot in the row sums)
    // per class: rows [row0[2c], row1[2c]) (hubs) and [row0[2c+1], row1[2c+1]) (the rest); nonzeros
    // [k0[i], k1[i]) of range i
    std::vector<int64_t> row0, row1, k0, k1;
    int32_t *long_rows = nullptr;  // rows over kLongChunks chunks, grouped by class
    std::vector<int64_t> long_off;  // class c's long rows: long_rows[long_off[c] .. long_off[c + 1])
};
constexpr int kLongChunks = 16;  // a row over this many chunks is combined by a warp

// Solve scratch, grown on demand and kept by the handle.
struct Workspace {
    int64_t cap_n = 0;      // nodes x right-hand sides the buffers hold
    int cap_graphs = 0;
    void *r = nullptr;      // residual (FP32 or FP64)
    void *h = nullptr;      // thresholds eps' s'
    void *da = nullptr;     // push increments (current)
    void *db = nullptr;     // push increments (second buffer)
    void *om = nullptr;     // per-node relaxation factor
    void *rsum = nullptr;   // single-vector sweep: row sums of the gathered increments, by row rank
    void *carry = nullptr;  // single-vector sweep: partial sum of the row that crosses each chunk's end
    int64_t cap_carry = 0;
    char *fdz = nullptr;     // frontier push: count, entries and steps set aside for the long scatter
    int64_t cap_fdz = 0;
    double *judge = nullptr;  // per-block residual and opinion sums of the warm-start judge
    int64_t cap_judge = 0;
    double *zhat = nullptr; // estimate of z' (FP64)
    double *sp = nullptr;   // s' = s + c_eff (FP64)
    double *sin = nullptr;  // caller's s, z0 or z staged on the device
    double *zout = nullptr; // unshifted result staged on the device
    double *r64 = nullptr;  // FP64 residual written by the certificate (frontier push state)
    float2 *zs = nullptr;   // zhat as FP32 pairs hi + lo for the certificate's off-diagonal sums
    double *gstat = nullptr;  // per graph/RHS: [c_eff, min s, resid_inf, resid_rel, z_inf, violators]
    Counters *ctr = nullptr;
    Counters *ctr_host = nullptr;  // pinned mirror
    unsigned long long *zmax = nullptr;  // max |zhat| before a certificate (ordered bits)
    double *gstat_host = nullptr;  // pinned mirror
    unsigned long long *status = nullptr;  // look-back tile status
    int64_t cap_status = 0;
    unsigned int *tile_ctr = nullptr;
    int32_t *list = nullptr;  // frontier list
    long long *count = nullptr;
    double *partial = nullptr;  // per-block partial sums (metrics)
    int64_t cap_partial = 0;
    int64_t sweep_parity = 0;   // sweeps launched on this handle; selects the increment buffers
    // captured batches of sweeps, per (precision, schedule); valid while gen == graph_gen
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t gkey[2][2] = {{-1, -1}, {-1, -1}};
    int gsweeps[2][2] = {{0, 0}, {0, 0}};
    int glaunch[2][2] = {{0, 0}, {0, 0}};
    cudaStream_t cap_stream = nullptr;
    int64_t gen = 0;            // bumped whenever buffers or work-item plans change
};

// Scratch of a multi-right-hand-side solve: node-major [n][k] arrays.
struct BatchWorkspace {
    int64_t cap = 0;   // n * k entries held
    int cap_k = 0;
    void *r = nullptr, *h = nullptr, *da = nullptr, *db = nullptr;
    void *z32 = nullptr;       // FP32 path: increments of the current pass, folded into zhat
    double *zhat = nullptr, *sp = nullptr, *sin = nullptr, *zout = nullptr;
    double *r64 = nullptr;     // FP64 residual written by the certificate
    int32_t *list = nullptr;   // frontier of (node, vector) entries, n * k capacity
    void *om = nullptr;        // per node
    double *gstat = nullptr;   // per right-hand side, kGs words
    double *gstat_host = nullptr;
    double *partk = nullptr;   // per long-row chunk and right-hand side (two words: hi, lo)
    int64_t cap_partk = 0;
    unsigned int *tick = nullptr;  // per colour class: next tile, retired warps
    int64_t cap_tick = 0;
    int depth = 0;                 // gathers in flight per warp: 4 or 8 per-lane loads, 0 = bulk copies (FP32)
};

}  // namespace fj

struct fj_graph {
    int device = 0;
    int directed = 0;
    int ngraphs = 1;
    fj::DevCSR csr;
    // transposed CSR (directed graphs): row v lists u with a_uv > 0
    int64_t *tptr = nullptr;
    int32_t *tcol = nullptr;
    float *tw = nullptr;
    std::vector<int64_t> node_off;     // host, ngraphs + 1
    int64_t *node_off_d = nullptr;
    fj::Colouring colr;
    fj::ItemPlan wplan_csr, wplan_pcsr;  // warp-tile items (certificate, batch sweep, network)
    fj::ChunkPlan cplan_csr, cplan_pcsr;  // chunk plans (single-vector sweep)
    fj::Workspace ws;
    fj::BatchWorkspace bws;
    fj::SortScratch sort;
    int *err = nullptr;      // device error word
    int *err_host = nullptr; // pinned mirror
};

namespace fj {

// fj_graph.cu
fj_status graph_finish(fj_graph *g, cudaStream_t st);
fj_status build_blocks(DevCSR &c, const std::vector<int64_t> &seg_rows, Workspace &ws, int *err,
                       cudaStream_t st, TileKind kind);
fj_status ensure_colouring(fj_graph *g, int palette, cudaStream_t st);
fj_status ensure_ptranspose(fj_graph *g, cudaStream_t st);
// fj_solve.cu
fj_status plain_items(fj_graph *g, cudaStream_t st, const ItemPlan **out);
fj_status ws_status(Workspace &ws, int64_t tiles);
fj_status read_dev_error(fj_graph *g, cudaStream_t st);
void dev_free(void *p);
void chunk_plan_free(ChunkPlan &cp);

}  // namespace fj
