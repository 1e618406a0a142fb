// Host-side plan tables of the fused H.v (kernels in ed_hv2_kernel.cuh and
// ed_hv2c_kernel.cuh): plain C++, no CUDA, so that they also build and run where no GPU is.
#pragma once

#include <stdint.h>

#include <vector>

#include "ed.h"

namespace ed {

constexpr uint32_t kTargetMask = 0x3FFFFFFFu;  // hop entry: target rank in bits 0..29
constexpr uint32_t kSignBit = 0x80000000u;     // hop entry: bit 31 = negative fermion sign

// Thread-local error message behind ed_last_error().
void set_error(const char* fmt, ...);

// Down-hop tables of one species for one kernel geometry (V columns per thread, G slots per
// bank group). Columns p are the down states ordered by hop count (most first), then by
// +1-hop count, then by rank: p = pos[rank]. Per chunk of 32 V columns the table rows
// [0, kpn[2c]) hold the +1 hops and [kpn[2c], kpn[2c] + kpn[2c+1]) the -1 hops (complex
// tables: all hops in the first kpn[2c] rows, the sign in the amplitude index), each
// column's hops in the order schedule_gathers gives them; an entry is the shared-memory
// slot of the hop's target, or one of the zero slots ld .. ld + G - 1 for padding.
struct DownTables {
  int V = 0, G = 0, ld = 0, rows = 0;
  bool cplx = false;              // 32-bit entries slot | signed amplitude index << 16
  std::vector<uint16_t> tab;      // [rows][ld] (real tables)
  std::vector<uint32_t> tab32;    // [rows][ld] (complex tables)
  std::vector<uint8_t> kpn;       // [2 * chunks]: +1 rows, -1 rows
  std::vector<uint8_t> lo;        // [ld] slot of column p inside its aligned group of G
  std::vector<uint32_t> pad;      // [ld] down bit string by column (0 on pads)
  std::vector<int32_t> pos;       // [n] column of each down rank
};

// Build the tables from the species' host tables: hop [mh][n] (target | sign << 31, entries
// >= n after masking are padding), hopa [mh][n] amplitude numbers or null, bits [n].
// ld = n rounded up to 32. ED_ERR_ARG (message set) when a column has more than 255 hops
// of one sign or the geometry is invalid.
ed_status build_down_tables(const int32_t* hop, const int32_t* hopa, const uint32_t* bits,
                            int64_t n, int mh, int ld, int V, int G, bool cplx, DownTables& out);

// Split-row tables (two slices of the down states by the occupation of one site, for rows
// longer than shared memory): see build_split_tables.
struct SplitTables {
  int V = 0, G = 0, site = 0, ld = 0, rows = 0, xrows = 0;
  int cstart[3] = {0, 0, 0};     // slice s: columns [cstart[s], cstart[s+1])
  std::vector<uint16_t> tab;     // [rows][ld] in-slice slots (zero slots ld_s .. ld_s + G - 1)
  std::vector<uint16_t> xtab;    // [xrows][ld] target column inside the other slice
  std::vector<uint8_t> kpn;      // [4 * chunks]: in-slice +1, -1 rows; cross +1, -1 rows
  std::vector<uint8_t> lo;       // [ld] slot of column p within its aligned group of G
  std::vector<uint32_t> pad;     // [ld] down bit string by column (0 on pads)
  std::vector<int32_t> pos;      // [n] column of each down rank
};

ed_status build_split_tables(const int32_t* hop, const uint32_t* bits, int64_t n, int mh, int V,
                             int G, int site, SplitTables& out);

}  // namespace ed
