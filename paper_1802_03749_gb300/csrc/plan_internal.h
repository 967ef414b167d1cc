// Internal plan representation shared by the host planner (plan.cpp) and
// the device glue (loops_*.cu).  Not part of the C ABI.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/meshloop.h"

struct mp_block_desc {          // one thread block of a HIER plan (32 bytes)
    int32_t item_start;         // first iteration (plan numbering)
    int32_t nitems;             // working threads of the block (<= S)
    int32_t ncolors;            // thread colours of the block
    int32_t pad;
    int32_t fp_start[MP_MAX_TOSETS];  // offset of the footprint list per to-set slot in the
                                      // concatenation of all slots' lists (slot 0 first)
    int32_t fp_count[MP_MAX_TOSETS];  // footprint size per to-set slot
};

struct mp_map_info {
    int32_t to_set;
    int32_t arity;
    int32_t written;
    int32_t slot;               // to-set slot (0..ntosets-1)
    int64_t to_size;
    std::vector<int32_t> idx;   // plan numbering, from_size x arity
};

struct mp_device_tables {
    int device = -1;
    mp_block_desc *desc = nullptr;
    uint16_t *lmap = nullptr;   // from_size x lmap_stride local indices (HIER)
    int32_t *fp = nullptr;      // all footprint lists, slot-major
    uint8_t *tcolor = nullptr;  // thread colour per iteration (HIER)
    uint16_t *gat = nullptr;    // HIER: block-local inverse of the written maps
    int32_t *color_off = nullptr;  // HIER: block range of each colour (persistent launches)
    unsigned *bar = nullptr;       // HIER: persistent launches: grid-barrier arrivals, then one
                                   // block counter per colour (ncolors + 1 words)
    int32_t *map[MP_MAX_MAPS] = {nullptr, nullptr, nullptr, nullptr};  // GLOBAL / ATOMIC / TWOSTEP
    int32_t *inv_off = nullptr;  // TWOSTEP: written to-set point -> range of inv_idx
    int32_t *inv_idx = nullptr;  // TWOSTEP: item * arity + slot, sorted by (point, item, slot)
    void *scratch = nullptr;     // TWOSTEP: per-(item, slot) increments
    size_t scratch_bytes = 0;
    void *host_io = nullptr;     // loop_res_calc_host: device buffers, copy streams (host_io.cu)
    int64_t bytes = 0;
};

struct mp_plan {
    int64_t from_size = 0;
    mp_plan_opts opts{};
    int32_t nmaps = 0;
    mp_map_info maps[MP_MAX_MAPS];
    int32_t ntosets = 0;
    int32_t toset_id[MP_MAX_TOSETS] = {0, 0};
    int64_t toset_size[MP_MAX_TOSETS] = {0, 0};

    std::vector<int32_t> perm_from;                 // new_to_old
    std::vector<int32_t> perm_to[MP_MAX_TOSETS];    // new_to_old per slot

    int32_t nblocks = 0;
    std::vector<int32_t> block_offsets;   // nblocks + 1
    std::vector<int32_t> block_color;     // nblocks
    int32_t ncolors = 0;                  // block colours (HIER) / iteration colours (GLOBAL)
    std::vector<int32_t> color_offsets;   // ncolors + 1: blocks (HIER) or iterations (GLOBAL)
    std::vector<uint8_t> thread_color;    // from_size
    std::vector<int32_t> block_ncolors;   // nblocks

    // TWOSTEP inverse of the written map
    int32_t inv_map = -1;
    std::vector<int32_t> inv_off, inv_idx;

    // HIER footprints
    std::vector<int32_t> fp_offsets[MP_MAX_TOSETS];  // nblocks + 1
    std::vector<int32_t> fp_ids[MP_MAX_TOSETS];
    // block-local inverse of the written maps, one row of gat_w entries per
    // point of the concatenated footprint lists: local iteration * 16 + map
    // slot of each increment, ascending, padded with 0xFFFF (gat_w 0: none)
    int32_t gat_w = 0;
    std::vector<uint16_t> gat_tab;
    int32_t lmap_stride = 0;              // padded slot count per iteration (4 or 8 or 16)
    std::vector<uint16_t> lmap;           // from_size x lmap_stride
    std::vector<mp_block_desc> desc;

    mp_plan_stats stats{};
    mp_device_tables dev;
};

// Implemented in loops_common.cu: frees the device tables of a plan.
void mp_plan_free_device(mp_plan *plan);
