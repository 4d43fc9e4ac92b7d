// Device-side program layout, cache and sampling entry points (device.cu).
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "program.h"

namespace tsim {

struct SampleArgs {
  uint64_t shots = 0, seed = 0, shot_offset = 0;
  uint64_t* meas = nullptr;
  uint64_t* det = nullptr;
  uint64_t* obs = nullptr;
  uint8_t* accept = nullptr;
};

// Tables with at least this many terms (after merging equal factor lists)
// use the bit-sliced warp-cooperative layout when their factors allow it
// (measured: 4 beats 2, 16 and 64 on the colour-code and mirror workloads).
constexpr int64_t kDefaultSlicedMin = 4;

// Byte offsets of the sections of the packed device tables (256-byte aligned)
struct DeviceLayout {
  size_t o_grp = 0, o_gmem = 0, o_gT = 0;  // geometric-gap noise groups, members, gap tables
  size_t o_cf = 0, o_ffi = 0, o_ffa = 0;   // chain float flags; arbitrary-angle factors (parity, angle)
  size_t o_tc = 0;                          // per table: the precomputed value of a constant table
  size_t o_dmk = 0, o_omk = 0, o_dcs = 0, o_ocs = 0;  // measurement mode: detector / observable X-masks, constants
  size_t o_ch = 0, o_t0 = 0, o_thr = 0, o_sig = 0, o_out = 0, o_om = 0, o_cn = 0, o_tab = 0, o_par = 0, o_pidx = 0,
         o_cls = 0, o_fidx = 0, o_finc = 0, o_fco = 0, o_seg = 0, o_sb = 0, o_row = 0, o_dmo = 0, o_dmi = 0, o_omo = 0,
         o_omi = 0, total = 0;
  int W = 1;
  int n_ent = 0;            // output entries (runs of single-bit outputs merged)
  uint64_t runs = 0, run_outputs = 0;  // runs and the outputs they cover
  uint32_t sl_par_max = 0;  // largest parity list of a bit-sliced table
  uint32_t sl_rows_max = 0; // most operation rows of a staged batch
  int sl_par = 0;           // shared 32-bit words per warp for parity words (0: no sliced table)
  int sl_rb = 0;            // shared 32-bit words of one row staging buffer (0: none)
  // statistics of the packed tables
  uint64_t classes = 0;     // stabilizer terms after merging terms with equal factor lists
  uint64_t class_factors = 0;
  uint64_t parities = 0;    // distinct factor parities over all tables
  std::vector<uint64_t> table_classes, table_class_factors, table_parities;  // per table
  // per table: layout (0 scalar, 1 basis, 2 bit-sliced), and for sliced
  // tables the batches of 32 terms, padded operation rows and real operations
  std::vector<uint64_t> table_mode, table_batches, table_rows, table_ops;
  std::vector<uint64_t> table_work32;       // sliced: integer lane-operations of one warp (32 shots)
  std::vector<uint64_t> table_work32_real;  // the same without row and lane padding
};

// Host-side packed tables of one program, built once when the program is
// compiled or loaded.  status != TSIM_OK when the program cannot run on the
// device (message says why); sampling then fails with that status.
struct DeviceTables {
  std::vector<unsigned char> blob;
  DeviceLayout layout;
  tsim_status status = TSIM_OK;
  std::string message;
  // the packing arguments, as given to prepare_device_tables
  int64_t sliced_min = kDefaultSlicedMin;
  int stage_rows = -1, seg_par = 0;
};

// Sliced batches with at most this many operation rows are staged through
// shared memory by bulk copies.  Off by default: the staging buffers cost
// resident warps, and on the colour-code T-check the rows read through L1
// were faster (1.08e7 against 8.8e6 shots/s).
constexpr int kDefaultStageRows = 0;

// Sliced tables are split into segments of consecutive terms whose parity
// words (two reserved) fit this many 32-bit words of shared memory per warp.
constexpr int kDefaultSegmentParities = 1536;

// Pack the device tables; sliced_min < 0 disables the bit-sliced layout;
// stage_rows: largest staged batch (0: read rows from global memory, < 0:
// the default); seg_par: parity words per segment (<= 0: the default).
void prepare_device_tables(Program& p, int64_t sliced_min = kDefaultSlicedMin, int stage_rows = -1,
                           int seg_par = 0);
// Host emulation of every bit-sliced table of the packed program, 32 random
// per-shot vectors X per round, compared exactly with the host evaluation of
// the same table; fails with TSIM_ERR_INTERNAL on any difference.
void selftest_sliced(const Program& p, uint64_t seed, int rounds);
void device_sample(const Program& p, const SampleArgs& a, void* stream);
// tsim_sample without device allocation: the tables go into the library's
// fixed static device array (see tsim_sample_noalloc).
void device_sample_noalloc(const Program& p, const SampleArgs& a, void* stream);
// tsim_sample plus a copy of every table evaluation of the chosen shots
// (indices within the launch): per shot, per evaluation (chain
// normalisations, then random outputs in order), [table, c0, c1, c2, c3,
// sqrt2 exponent, X words (x_words)].  Synchronises the stream.
void device_sample_debug(const Program& p, const SampleArgs& a, const uint64_t* dump_shots, int n_dump,
                         int64_t* h_dump, void* stream);
void device_sample_batch(const Program* const* progs, int n, const SampleArgs* args, void* stream);

struct BatchPlan;
BatchPlan* batch_create(const Program* const* progs, int n, const SampleArgs* args, int autotune);
void batch_launch(BatchPlan* b, void* stream);
void batch_free(BatchPlan* b);
void batch_info(const BatchPlan* b, int64_t out[7]);
void device_sync(void* stream);
void device_release(DeviceProgram* d);

// exact monomial form of a Clifford factor value: value = 0 or sqrt2^s w^j
bool monomial_of(const ZW& v, int* zero, int* s, int* j);

}  // namespace tsim
