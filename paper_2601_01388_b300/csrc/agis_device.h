// Definitions that the sampler kernels read (csrc/sample.cu): launch-shape
// constants, the compiled query, work items and the views of the graph and of the
// per-trial outputs.  Host-only runtime state is in agis_internal.h.
#pragma once

#include <stdint.h>

#include "../../include/agis.h"

namespace agis {

constexpr int kMaxK = 8;
#ifndef AGIS_TILE
#define AGIS_TILE 256
#endif
constexpr int kTile = AGIS_TILE;     // trials per work item (one CTA at a time)
static_assert(kTile >= 32 && kTile <= 1024 && (kTile & (kTile - 1)) == 0, "tile: power of two in [32, 1024]");
// A work item covers 1..kMaxSpan consecutive tiles of one query; each tile keeps its
// own fixed-order reduction and output slot, so results never depend on the span.
constexpr int kMaxSpan = 4;
constexpr int kBlock = 256;          // threads per CTA of the sampler
constexpr int kWarps = kBlock / 32;
constexpr uint64_t kStreamTrial = 1; // Philox counter word 2 of a trial draw
constexpr uint64_t kStreamCC = 2;    // ... of a clustering-coefficient probe

// One step of a compiled query as the sampler kernel reads it.
struct DevStep {
    int32_t nb;                 // |B[i]|: number of backward neighbours
    int8_t approx;              // 1: draw with the f_approx weight table (D(i) chose f_approx and
                                // the weights are not all equal on S_tau); 0: by position / degree
    int8_t dapprox;             // D(i) itself (1 = f_approx); only the survey's sector count reads it
    int8_t inc;                 // backward set = previous step's plus the previous vertex
    int8_t rp_mode;             // pref for |B| = 1: 0 none, 1 per-row prefix of every row,
                                // 2 prefix of high-degree rows only (located by rp_base)
    int8_t back[kMaxK];         // step indices of the backward neighbours
    const uint64_t *q;          // quantised f_approx weight per vertex (approx only)
    const uint64_t *pref;       // step 0: inclusive prefix over vertices; |B| = 1: row prefix
};

constexpr int32_t kFlagAnchor = 1;   // DevQuery::flags: anchor draw on several-backward steps
constexpr int32_t kFlagPlainLists = 2;  // DevQuery::flags: no candidate-list step weighs its survivors

struct DevQuery {
    int32_t k;
    int32_t flags;
    uint64_t seed;
    uint64_t W1;                // total step-1 weight (f_approx sum or nnz)
    DevStep step[kMaxK];
};

// Words of one tile's output (AGIS_TILE_WORDS): hits, model sectors, bits of sum X,
// bits of sum X^2, streamed part of the model sectors, survey-count sectors.
constexpr int kTileWords = AGIS_TILE_WORDS;

// A work item: `count` trials (at most kMaxSpan tiles) of query `query` starting at
// trial `first`; the sums of its t-th tile go to out[kTileWords*(slot+t) ...].
struct WorkItem {
    uint32_t query;
    uint32_t count;
    uint64_t first;
    uint64_t slot;
};

// Where a dump launch writes per-trial records (index = trial - dump_first).
struct DumpView {
    int32_t *emb;
    uint8_t *hit;
    double *x;
    uint64_t *sectors;          // 3 words per trial: model total, its streamed part, survey count
    uint64_t first;
};

// Per-trial outputs of a scatter launch (see scatter_kernel), indexed by the launch's
// item * kTile + trial within the tile.
struct ScatterView {
    double *x;
    uint8_t *hit;
    uint64_t *sec;              // 3 words per trial: sectors, streamed, survey
};

struct GraphView {
    const int64_t *off;
    const int32_t *cols;
    int64_t nv;
    int64_t nnz;
    const int32_t *hub_id;      // per vertex: index of its neighbour bitmap, -1 if none
    const uint32_t *hub_bits;   // bitmaps, hub_words 32-bit words each
    int64_t hub_words;
    const int64_t *rp_base;     // per vertex: start of its row in partial row-prefix tables, -1 if none
};

}  // namespace agis
