// extern "C" boundary: argument checks, exception -> status conversion.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>

#include "circuit.h"
#include "cutnet.h"
#include "device.h"
#include "program.h"
#include "zx.h"

#include <complex>

#include <cuda_runtime.h>

namespace {

thread_local char g_last_error[1024];

template <class F>
tsim_status guard(F&& f) {
  try {
    f();
    return TSIM_OK;
  } catch (const tsim::Error& e) {
    tsim::set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    tsim::set_last_error("host allocation failed");
    return TSIM_ERR_OOM;
  } catch (const std::exception& e) {
    tsim::set_last_error(e.what());
    return TSIM_ERR_INTERNAL;
  }
}

const tsim::Program& prog_of(const tsim_program* p) {
  if (!p || !p->p) tsim::fail(TSIM_ERR_ARG, "NULL program");
  return *p->p;
}

}  // namespace

tsim::Program::~Program() {
  tsim::device_release(dev);
  delete devtab;
}

void tsim::set_last_error(const char* msg) { std::snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

extern "C" {

const char* tsim_last_error(void) { return g_last_error; }

tsim_status tsim_compile(const char* text, size_t len, const tsim_compile_opts* opts, tsim_program** out) {
  return guard([&] {
    if (!text || !out) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    tsim_compile_opts o{};
    o.mode = TSIM_MODE_DETECTORS;
    o.decomp = TSIM_DECOMP_HEURISTIC;
    o.chi_budget = 0;
    o.channel_reduction = 1;
    o.total_budget = 0;
    if (opts) o = *opts;
    if (o.mode != TSIM_MODE_DETECTORS && o.mode != TSIM_MODE_MEASUREMENTS) tsim::fail(TSIM_ERR_ARG, "bad mode");
    if (o.decomp < 0 || o.decomp > 4) tsim::fail(TSIM_ERR_ARG, "bad decomposition policy");
    tsim::Program* p = tsim::compile_program(std::string(text, len), o);
    *out = new tsim_program{p};
  });
}

tsim_status tsim_program_info(const tsim_program* prog, tsim_program_info_t* out) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!out) tsim::fail(TSIM_ERR_ARG, "NULL info");
    std::memset(out, 0, sizeof *out);
    out->mode = p.mode;
    out->num_qubits = p.nq;
    out->num_measurements = p.nmeas;
    out->num_detectors = p.ndet;
    out->num_observables = p.nobs;
    out->num_error_bits = p.E;
    out->num_channels = (int)p.channels.size();
    out->num_f = p.nf;
    out->num_random = p.nr;
    out->num_outputs = (int)p.outputs.size();
    out->num_chains = (int)p.chain_norm.size();
    out->num_tables = (int)p.tables.size();
    out->x_words = p.W;
    for (const auto& t : p.tables) {
      out->total_terms += t.terms.size();
      out->max_terms = std::max<uint64_t>(out->max_terms, t.terms.size());
      for (const auto& tm : t.terms) out->max_factors = std::max(out->max_factors, (int)tm.f.size());
    }
    out->meas_words = (p.nmeas + 63) / 64;
    out->det_words = (p.ndet + 63) / 64;
    out->obs_words = (p.nobs + 63) / 64;
    if (p.devtab) {
      out->device_classes = p.devtab->layout.classes;
      out->device_parities = p.devtab->layout.parities;
      out->device_status = p.devtab->status;
    }
  });
}

tsim_status tsim_program_table_terms(const tsim_program* prog, int t, uint64_t* terms) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!terms || t < 0 || t >= (int)p.tables.size()) tsim::fail(TSIM_ERR_ARG, "bad table index");
    *terms = p.tables[(size_t)t].terms.size();
  });
}

tsim_status tsim_program_table_stats(const tsim_program* prog, int t, uint64_t* terms, uint64_t* factors) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!terms || !factors || t < 0 || t >= (int)p.tables.size()) tsim::fail(TSIM_ERR_ARG, "bad table index");
    *terms = p.tables[(size_t)t].terms.size();
    *factors = 0;
    for (const auto& tm : p.tables[(size_t)t].terms) *factors += tm.f.size();
  });
}

tsim_status tsim_program_device_table_stats(const tsim_program* prog, int t, uint64_t out[3]) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!out || t < 0 || t >= (int)p.tables.size()) tsim::fail(TSIM_ERR_ARG, "bad table index");
    if (!p.devtab || p.devtab->status != TSIM_OK) tsim::fail(TSIM_ERR_ARG, "program has no device tables");
    const auto& L = p.devtab->layout;
    out[0] = L.table_classes[(size_t)t];
    out[1] = L.table_class_factors[(size_t)t];
    out[2] = L.table_parities[(size_t)t];
  });
}

tsim_status tsim_program_set_table_layout(tsim_program* prog, int64_t sliced_min_terms, int32_t stage_rows,
                                          int32_t segment_parities) {
  return guard([&] {
    tsim::Program& p = const_cast<tsim::Program&>(prog_of(prog));
    tsim::device_release(p.dev);  // the uploaded copy of the old layout
    p.dev = nullptr;
    tsim::prepare_device_tables(p, sliced_min_terms, stage_rows, segment_parities);
    if (p.devtab->status != TSIM_OK) tsim::fail(p.devtab->status, p.devtab->message);
  });
}

tsim_status tsim_program_device_table_layout(const tsim_program* prog, int t, uint64_t out[6]) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!out || t < 0 || t >= (int)p.tables.size()) tsim::fail(TSIM_ERR_ARG, "bad table index");
    if (!p.devtab || p.devtab->status != TSIM_OK) tsim::fail(TSIM_ERR_ARG, "program has no device tables");
    const auto& L = p.devtab->layout;
    out[0] = L.table_mode[(size_t)t];
    out[1] = L.table_batches[(size_t)t];
    out[2] = L.table_rows[(size_t)t];
    out[3] = L.table_ops[(size_t)t];
    out[4] = L.table_work32[(size_t)t];
    out[5] = L.table_work32_real[(size_t)t];
  });
}

tsim_status tsim_program_device_output_stats(const tsim_program* prog, uint64_t out[3]) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!out) tsim::fail(TSIM_ERR_ARG, "NULL output array");
    if (!p.devtab || p.devtab->status != TSIM_OK) tsim::fail(TSIM_ERR_ARG, "program has no device tables");
    const auto& L = p.devtab->layout;
    out[0] = (uint64_t)L.n_ent;
    out[1] = L.runs;
    out[2] = L.run_outputs;
  });
}

tsim_status tsim_sample(const tsim_program* prog, uint64_t shots, uint64_t seed, uint64_t shot_offset,
                        uint64_t* d_meas, uint64_t* d_det, uint64_t* d_obs, uint8_t* d_accept,
                        void* cuda_stream) {
  return guard([&] {
    tsim::SampleArgs a;
    a.shots = shots;
    a.seed = seed;
    a.shot_offset = shot_offset;
    a.meas = d_meas;
    a.det = d_det;
    a.obs = d_obs;
    a.accept = d_accept;
    tsim::device_sample(prog_of(prog), a, cuda_stream);
  });
}

// For callers that cannot allocate device memory: same records as
// tsim_sample, with the program's tables in the library's fixed static
// device array (device.cu); errors come back as a status, as everywhere.
tsim_status tsim_sample_noalloc(const tsim_program* prog, uint64_t shots, uint64_t seed, uint64_t shot_offset,
                                uint64_t* d_meas, uint64_t* d_det, uint64_t* d_obs, uint8_t* d_accept,
                                void* cuda_stream) {
  return guard([&] {
    tsim::SampleArgs a;
    a.shots = shots;
    a.seed = seed;
    a.shot_offset = shot_offset;
    a.meas = d_meas;
    a.det = d_det;
    a.obs = d_obs;
    a.accept = d_accept;
    tsim::device_sample_noalloc(prog_of(prog), a, cuda_stream);
  });
}

tsim_status tsim_debug_sample(const tsim_program* prog, uint64_t shots, uint64_t seed, uint64_t shot_offset,
                              uint64_t* d_meas, uint64_t* d_det, uint64_t* d_obs, uint8_t* d_accept,
                              const uint64_t* dump_shots, int n_dump, int64_t* h_dump, void* cuda_stream) {
  return guard([&] {
    tsim::SampleArgs a;
    a.shots = shots;
    a.seed = seed;
    a.shot_offset = shot_offset;
    a.meas = d_meas;
    a.det = d_det;
    a.obs = d_obs;
    a.accept = d_accept;
    tsim::device_sample_debug(prog_of(prog), a, dump_shots, n_dump, h_dump, cuda_stream);
  });
}

tsim_status tsim_program_set_noise_sampling(tsim_program* prog, int mode) {
  return guard([&] {
    tsim::Program& p = const_cast<tsim::Program&>(prog_of(prog));
    tsim::device_release(p.dev);  // the uploaded copy of the old layout
    p.dev = nullptr;
    // re-pack with the table layout the program already has
    int64_t smin = tsim::kDefaultSlicedMin;
    int stage = -1, seg = 0;
    if (p.devtab) {
      smin = p.devtab->sliced_min;
      stage = p.devtab->stage_rows;
      seg = p.devtab->seg_par;
    }
    tsim::set_noise_sampling(p, mode);
    tsim::prepare_device_tables(p, smin, stage, seg);
    if (p.devtab->status != TSIM_OK) tsim::fail(p.devtab->status, p.devtab->message);
  });
}

tsim_status tsim_program_device_bytes(const tsim_program* prog, uint64_t* bytes) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!bytes) tsim::fail(TSIM_ERR_ARG, "NULL output");
    if (!p.devtab || p.devtab->status != TSIM_OK) tsim::fail(TSIM_ERR_ARG, "program has no device tables");
    *bytes = p.devtab->layout.total;
  });
}

tsim_status tsim_program_noise_info(const tsim_program* prog, double out[4]) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!out) tsim::fail(TSIM_ERR_ARG, "NULL output array");
    double est[2];
    tsim::noise_word_estimate(p, est);
    out[0] = p.noise_mode;
    out[1] = (double)p.groups.size();
    out[2] = est[0];
    out[3] = est[1];
  });
}

tsim_status tsim_sample_host(const tsim_program* prog, uint64_t shots, uint64_t seed, uint64_t shot_offset,
                             uint64_t* h_meas, uint64_t* h_det, uint64_t* h_obs, uint8_t* h_accept,
                             void* cuda_stream) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (p.mode == TSIM_MODE_DETECTORS && h_meas) tsim::fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
    if (shots == 0) return;
    const size_t mw = (size_t)(p.nmeas + 63) / 64, dw = (size_t)(p.ndet + 63) / 64, ow = (size_t)(p.nobs + 63) / 64;
    // bytes of one shot's records
    const size_t row = (h_meas ? mw * 8 : 0) + (h_det ? dw * 8 : 0) + (h_obs ? ow * 8 : 0) + (h_accept ? 1 : 0);
    // chunks of at least 2^18 shots (at most 8): the copies of one chunk
    // overlap the sampling of the next
    const uint64_t nchunk = std::max<uint64_t>(1, std::min<uint64_t>(8, shots >> 18));
    const uint64_t chunk = (shots + nchunk - 1) / nchunk;
    // per host thread and device: two staging buffers, a copy stream and
    // events, grown as needed and kept until the process exits
    struct Staging {
      int device = -1;
      unsigned char* d = nullptr;
      size_t size = 0;
      cudaStream_t copy = nullptr;
      cudaEvent_t done[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    };
    static thread_local Staging st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) tsim::fail(TSIM_ERR_CUDA, "cudaGetDevice failed");
    const size_t half = ((chunk * row + 255) & ~(size_t)255) + 256;
    if (st.device != dev) {  // resources of another device are left as they are
      st = Staging();
      st.device = dev;
      if (cudaStreamCreateWithFlags(&st.copy, cudaStreamNonBlocking) != cudaSuccess)
        tsim::fail(TSIM_ERR_CUDA, "cudaStreamCreate of the copy stream failed");
      for (int b = 0; b < 2; ++b)
        if (cudaEventCreateWithFlags(&st.done[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&st.freed[b], cudaEventDisableTiming) != cudaSuccess)
          tsim::fail(TSIM_ERR_CUDA, "cudaEventCreate failed");
    }
    if (st.size < 2 * half) {
      if (st.copy) cudaStreamSynchronize(st.copy);
      if (st.d) cudaFree(st.d);
      st.d = nullptr;
      st.size = 0;
      cudaError_t e = cudaMalloc(&st.d, 2 * half);
      if (e != cudaSuccess) tsim::fail(TSIM_ERR_OOM, std::string("cudaMalloc staging: ") + cudaGetErrorString(e));
      st.size = 2 * half;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    auto ck = [](cudaError_t ce, const char* what) {
      if (ce != cudaSuccess) tsim::fail(TSIM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(ce));
    };
    // copies left by a call that failed part-way must not race with this one
    ck(cudaStreamSynchronize(st.copy), "cudaStreamSynchronize");
    for (uint64_t k = 0; k < nchunk; ++k) {
      const uint64_t first = k * chunk;
      if (first >= shots) break;
      const uint64_t n = std::min<uint64_t>(chunk, shots - first);
      const int b = (int)(k & 1);
      unsigned char* d = st.d + (size_t)b * half;
      if (k >= 2) ck(cudaStreamWaitEvent(s, st.freed[b], 0), "cudaStreamWaitEvent");  // buffer b copied out
      const size_t bm = h_meas ? n * mw * 8 : 0, bd = h_det ? n * dw * 8 : 0, bo = h_obs ? n * ow * 8 : 0;
      tsim::SampleArgs a;
      a.shots = n;
      a.seed = seed;
      a.shot_offset = shot_offset + first;
      a.meas = h_meas ? (uint64_t*)d : nullptr;
      a.det = h_det ? (uint64_t*)(d + bm) : nullptr;
      a.obs = h_obs ? (uint64_t*)(d + bm + bd) : nullptr;
      a.accept = h_accept ? (uint8_t*)(d + bm + bd + bo) : nullptr;
      tsim::device_sample(p, a, cuda_stream);
      ck(cudaEventRecord(st.done[b], s), "cudaEventRecord");
      ck(cudaStreamWaitEvent(st.copy, st.done[b], 0), "cudaStreamWaitEvent");
      auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (bytes) ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st.copy), "cudaMemcpyAsync");
      };
      cp(h_meas ? h_meas + first * mw : nullptr, a.meas, bm);
      cp(h_det ? h_det + first * dw : nullptr, a.det, bd);
      cp(h_obs ? h_obs + first * ow : nullptr, a.obs, bo);
      cp(h_accept ? h_accept + first : nullptr, a.accept, h_accept ? n : 0);
      ck(cudaEventRecord(st.freed[b], st.copy), "cudaEventRecord");
    }
    ck(cudaStreamSynchronize(st.copy), "cudaStreamSynchronize");
    tsim::device_sync(cuda_stream);
  });
}

struct tsim_batch {
  tsim::BatchPlan* b;
};

namespace {

std::vector<tsim::SampleArgs> batch_args(int n, const uint64_t* shots, const uint64_t* seeds,
                                         const uint64_t* shot_offsets, uint64_t* const* d_meas,
                                         uint64_t* const* d_det, uint64_t* const* d_obs,
                                         uint8_t* const* d_accept) {
  if (n < 0 || (n > 0 && (!shots || !seeds))) tsim::fail(TSIM_ERR_ARG, "bad batch arguments");
  std::vector<tsim::SampleArgs> as((size_t)n);
  for (int i = 0; i < n; ++i) {
    as[(size_t)i].shots = shots[i];
    as[(size_t)i].seed = seeds[i];
    as[(size_t)i].shot_offset = shot_offsets ? shot_offsets[i] : 0;
    as[(size_t)i].meas = d_meas ? d_meas[i] : nullptr;
    as[(size_t)i].det = d_det ? d_det[i] : nullptr;
    as[(size_t)i].obs = d_obs ? d_obs[i] : nullptr;
    as[(size_t)i].accept = d_accept ? d_accept[i] : nullptr;
  }
  return as;
}

std::vector<const tsim::Program*> batch_progs(const tsim_program* const* progs, int n) {
  if (n > 0 && !progs) tsim::fail(TSIM_ERR_ARG, "NULL program array");
  std::vector<const tsim::Program*> ps((size_t)n);
  for (int i = 0; i < n; ++i) ps[(size_t)i] = &prog_of(progs[i]);
  return ps;
}

}  // namespace

tsim_status tsim_sample_batch(const tsim_program* const* progs, int n, const uint64_t* shots,
                              const uint64_t* seeds, const uint64_t* shot_offsets, uint64_t* const* d_meas,
                              uint64_t* const* d_det, uint64_t* const* d_obs, uint8_t* const* d_accept,
                              void* cuda_stream) {
  return guard([&] {
    auto as = batch_args(n, shots, seeds, shot_offsets, d_meas, d_det, d_obs, d_accept);
    auto ps = batch_progs(progs, n);
    tsim::device_sample_batch(ps.data(), n, as.data(), cuda_stream);
  });
}

tsim_status tsim_batch_create(const tsim_program* const* progs, int n, const uint64_t* shots,
                              const uint64_t* seeds, const uint64_t* shot_offsets, uint64_t* const* d_meas,
                              uint64_t* const* d_det, uint64_t* const* d_obs, uint8_t* const* d_accept,
                              int autotune, tsim_batch** out) {
  return guard([&] {
    if (!out) tsim::fail(TSIM_ERR_ARG, "NULL output");
    auto as = batch_args(n, shots, seeds, shot_offsets, d_meas, d_det, d_obs, d_accept);
    auto ps = batch_progs(progs, n);
    *out = new tsim_batch{tsim::batch_create(ps.data(), n, as.data(), autotune)};
  });
}

tsim_status tsim_batch_launch(tsim_batch* batch, void* cuda_stream) {
  return guard([&] {
    if (!batch || !batch->b) tsim::fail(TSIM_ERR_ARG, "NULL batch");
    tsim::batch_launch(batch->b, cuda_stream);
  });
}

tsim_status tsim_batch_info(const tsim_batch* batch, int64_t out[7]) {
  return guard([&] {
    if (!batch || !batch->b || !out) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    tsim::batch_info(batch->b, out);
  });
}

void tsim_batch_free(tsim_batch* batch) {
  if (!batch) return;
  tsim::batch_free(batch->b);
  delete batch;
}

tsim_status tsim_sync(void* cuda_stream) {
  return guard([&] { tsim::device_sync(cuda_stream); });
}

tsim_status tsim_eval_table(const tsim_program* prog, int t, const uint64_t* x, int64_t out_zw[4],
                            int32_t* sqrt2_exp) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!x || !out_zw || !sqrt2_exp) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    tsim::ZW v = tsim::eval_table_host(p, t, x);
    // reduce the exponent while every coefficient stays integral
    for (int i = 0; i < 4; ++i) {
      if (v.c[i] > INT64_MAX || v.c[i] < INT64_MIN) tsim::fail(TSIM_ERR_OVERFLOW_BOUND, "value exceeds int64");
      out_zw[i] = (int64_t)v.c[i];
    }
    *sqrt2_exp = v.k;
  });
}

tsim_status tsim_eval_table_float(const tsim_program* prog, int t, const uint64_t* x, double out[2]) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!x || !out) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    const std::complex<double> v = tsim::eval_table_host_c(p, t, x);
    out[0] = v.real();
    out[1] = v.imag();
  });
}

tsim_status tsim_raw_to_x(const tsim_program* prog, const uint8_t* e, uint64_t* x) {
  return guard([&] {
    const tsim::Program& p = prog_of(prog);
    if (!e || !x) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    std::memset(x, 0, (size_t)p.W * 8);
    int bit = 0;
    for (const auto& r : p.raw)
      for (int b = 0; b < r.nbits; ++b, ++bit)
        if (e[bit])
          for (int w = 0; w < p.W; ++w) x[w] ^= r.cols[(size_t)b][(size_t)w];
  });
}

tsim_status tsim_program_save(const tsim_program* prog, const char* path) {
  return guard([&] {
    if (!path) tsim::fail(TSIM_ERR_ARG, "NULL path");
    tsim::save_program(prog_of(prog), path);
  });
}

tsim_status tsim_program_load(const char* path, tsim_program** out) {
  return guard([&] {
    if (!path || !out) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    *out = new tsim_program{tsim::load_program(path)};
  });
}

void tsim_program_free(tsim_program* prog) {
  if (!prog) return;
  delete prog->p;
  delete prog;
}

tsim_status tsim_selftest_sliced(const tsim_program* prog, uint64_t seed, int rounds) {
  return guard([&] {
    if (rounds < 0) tsim::fail(TSIM_ERR_ARG, "negative rounds");
    tsim::selftest_sliced(prog_of(prog), seed, rounds);
  });
}

tsim_status tsim_selftest_rules(uint64_t seed, int iterations) {
  return guard([&] {
    std::mt19937_64 rng(seed);
    for (int it = 0; it < iterations; ++it) {
      const size_t np = 1 + rng() % 4;
      tsim::Graph g(np);
      int nv = 1 + (int)(rng() % 11);  // up to 11: groups of five odd spiders (Cat5) occur
      for (int v = 0; v < nv; ++v) {
        int l = (int)(rng() % 8);
        g.add_var(l);
        for (size_t q = 0; q < np; ++q)
          if (rng() % 3 == 0) g.P[(size_t)v].flip(q);
      }
      for (int a = 0; a < nv; ++a)
        for (int b = a + 1; b < nv; ++b)
          if (rng() % 2) g.toggle(a, b);
      g.s2 = (int)(rng() % 5) - 2;
      g.ph = (int)(rng() % 8);
      std::vector<tsim::ZW> want(1u << np);
      for (uint32_t pv = 0; pv < (1u << np); ++pv) {
        tsim::Bits b(np);
        for (size_t q = 0; q < np; ++q)
          if ((pv >> q) & 1) b.set(q);
        want[pv] = tsim::brute_value(g, b);
      }
      auto check = [&](const std::vector<tsim::Term>& terms, const char* what) {
        for (uint32_t pv = 0; pv < (1u << np); ++pv) {
          tsim::Bits b(np);
          for (size_t q = 0; q < np; ++q)
            if ((pv >> q) & 1) b.set(q);
          tsim::ZW s;
          for (const auto& t : terms) s = tsim::zw_add(s, tsim::term_value(t, b));
          tsim::ZW d = want[pv];
          for (auto& c : d.c) c = -c;
          if (!tsim::zw_add(s, d).zero())
            tsim::fail(TSIM_ERR_INTERNAL, std::string("rewrite self-test failed (") + what + ") at iteration " +
                                              std::to_string(it));
        }
      };
      for (int policy : {0, 4, 3, 2}) {
        std::vector<tsim::Term> terms;
        tsim::DecompStats st;
        tsim::decompose(g, policy, terms, st);
        check(terms, policy == 0 ? "heuristic" : policy == 4 ? "cat5" : policy == 3 ? "pairs" : "single cuts");
      }
      {
        // a score-ordered cut sequence (random scores, a forced first cut)
        // must give the same sum as any other order
        tsim::Graph h = g;
        for (int v = 0; v < h.n; ++v) h.uid[(size_t)v] = v;
        std::vector<double> scores((size_t)h.n);
        for (auto& x : scores) x = (double)(rng() % 1000);
        std::vector<tsim::Term> terms;
        tsim::DecompStats st;
        tsim::decompose(h, TSIM_DECOMP_LEARNED, terms, st, &scores, (int)(rng() % (uint64_t)std::max(1, h.n)));
        check(terms, "score order");
      }
      {
        // the same graph with arbitrary angles on some spiders: every policy
        // must reproduce the brute-force value in complex double
        tsim::Graph h = g;
        for (int v = 0; v < h.n; ++v)
          if (rng() % 3 == 0) h.set_angle(v, (double)(rng() % 1000) / 997.0);
        if (rng() % 2) h.fph = (double)(rng() % 1000) / 991.0;
        if (np > 0 && rng() % 2) {
          tsim::Bits a(np);
          a.set(rng() % np);
          h.add_factor_f((double)(rng() % 1000) / 983.0, a);
        }
        for (int policy : {0, 3, 2}) {
          std::vector<tsim::Term> terms;
          tsim::DecompStats st;
          tsim::decompose(h, policy, terms, st);
          for (uint32_t pv = 0; pv < (1u << np); ++pv) {
            tsim::Bits b(np);
            for (size_t q = 0; q < np; ++q)
              if ((pv >> q) & 1) b.set(q);
            std::complex<double> sum = 0.0;
            for (const auto& t : terms) sum += tsim::term_value_c(t, b);
            const std::complex<double> want = tsim::brute_value_c(h, b);
            if (std::abs(sum - want) > 1e-9 * (1.0 + std::abs(want)))
              tsim::fail(TSIM_ERR_INTERNAL, "rewrite self-test with arbitrary angles failed at iteration " +
                                                std::to_string(it));
          }
        }
      }
      // single steps on a copy: each must preserve the brute-force value
      tsim::Graph h = g;
      for (int v = 0; v < h.n; ++v) {
        if (!h.alive[(size_t)v]) continue;
        int l = h.lam[(size_t)v];
        if (l == 2 || l == 6) h.lcomp(v);
        else if ((l == 0 || l == 4) && h.degree(v) == 0) h.remove_isolated(v);
        else continue;
        for (uint32_t pv = 0; pv < (1u << np); ++pv) {
          tsim::Bits b(np);
          for (size_t q = 0; q < np; ++q)
            if ((pv >> q) & 1) b.set(q);
          tsim::ZW d = want[pv];
          for (auto& c : d.c) c = -c;
          if (!tsim::zw_add(tsim::brute_value(h, b), d).zero())
            tsim::fail(TSIM_ERR_INTERNAL, "single rewrite step changed the value at iteration " + std::to_string(it));
        }
      }
    }
  });
}

}  // extern "C"

namespace {

// Copies and checks a graph batch given through the C ABI.
tsim::cutnet::Batch make_batch(int n, const float* x, const int* rowptr, const int* col, const float* y,
                               int n_graphs, const int* goff, bool symmetric) {
  using tsim::fail;
  tsim::cutnet::Batch b;
  if (n < 0 || (n && (!x || !rowptr)) || n_graphs < 1 || (goff == nullptr && n_graphs != 1))
    fail(TSIM_ERR_ARG, "bad graph batch sizes or NULL arrays");
  b.n = n;
  b.X.assign(x, x + (size_t)n * TSIM_CUT_FEATURES);
  if (n) b.rowptr.assign(rowptr, rowptr + n + 1);
  else b.rowptr = {0};
  if (b.rowptr[0] != 0) fail(TSIM_ERR_ARG, "rowptr[0] must be 0");
  for (int i = 0; i < n; ++i)
    if (b.rowptr[(size_t)i + 1] < b.rowptr[(size_t)i]) fail(TSIM_ERR_ARG, "rowptr is not monotone");
  const int nnz = b.rowptr[(size_t)n];
  if (nnz && !col) fail(TSIM_ERR_ARG, "NULL col");
  b.col.assign(col ? col : nullptr, col ? col + nnz : nullptr);
  for (int c : b.col)
    if (c < 0 || c >= n) fail(TSIM_ERR_ARG, "neighbour id out of range");
  if (goff) b.goff.assign(goff, goff + n_graphs + 1);
  else b.goff = {0, n};
  if (b.goff.front() != 0 || b.goff.back() != n) fail(TSIM_ERR_ARG, "graph offsets must run from 0 to n");
  for (int g = 0; g < n_graphs; ++g)
    if (b.goff[(size_t)g + 1] < b.goff[(size_t)g]) fail(TSIM_ERR_ARG, "graph offsets are not monotone");
  if (y) b.y.assign(y, y + n);
  if (symmetric) {
    std::vector<std::vector<int>> adj((size_t)n);
    for (int v = 0; v < n; ++v) {
      for (int e = b.rowptr[(size_t)v]; e < b.rowptr[(size_t)v + 1]; ++e) {
        const int u = b.col[(size_t)e];
        if (u == v) fail(TSIM_ERR_ARG, "self loop in the adjacency");
        adj[(size_t)v].push_back(u);
      }
      std::sort(adj[(size_t)v].begin(), adj[(size_t)v].end());
      if (std::adjacent_find(adj[(size_t)v].begin(), adj[(size_t)v].end()) != adj[(size_t)v].end())
        fail(TSIM_ERR_ARG, "repeated edge in the adjacency");
    }
    for (int v = 0; v < n; ++v)
      for (int u : adj[(size_t)v])
        if (!std::binary_search(adj[(size_t)u].begin(), adj[(size_t)u].end(), v))
          fail(TSIM_ERR_ARG, "the adjacency is not symmetric");
    for (int g = 0; g < n_graphs; ++g)
      for (int v = b.goff[(size_t)g]; v < b.goff[(size_t)g + 1]; ++v)
        for (int u : adj[(size_t)v])
          if (u < b.goff[(size_t)g] || u >= b.goff[(size_t)g + 1]) fail(TSIM_ERR_ARG, "an edge joins two graphs");
  }
  return b;
}

}  // namespace

extern "C" {

int tsim_cut_num_params(void) { return tsim::cutnet::num_params(); }

tsim_status tsim_cut_init_params(uint64_t seed, float* params) {
  return guard([&] {
    if (!params) tsim::fail(TSIM_ERR_ARG, "NULL params");
    tsim::cutnet::init_params(seed, params);
  });
}

tsim_status tsim_cut_dataset(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget,
                             int max_candidates, const char* path) {
  return guard([&] {
    if (!path) tsim::fail(TSIM_ERR_ARG, "NULL path");
    tsim::cutnet::write_dataset(seed, n_graphs, t_min, t_max, budget, max_candidates, path);
  });
}

tsim_status tsim_cut_forward(const float* params, int n_nodes, const float* x, const int* rowptr,
                             const int* col, float* scores) {
  return guard([&] {
    if (!params || (n_nodes && !scores)) tsim::fail(TSIM_ERR_ARG, "NULL params or scores");
    tsim::cutnet::Batch b = make_batch(n_nodes, x, rowptr, col, nullptr, 1, nullptr, false);
    tsim::cutnet::forward(params, b, scores);
  });
}

tsim_status tsim_cut_loss_grad(const float* params, int n_nodes, const float* x, const int* rowptr,
                               const int* col, const float* y, int n_graphs, const int* graph_off,
                               float* loss, float* grad) {
  return guard([&] {
    if (!params || !grad || !loss || (n_nodes && !y)) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    tsim::cutnet::Batch b = make_batch(n_nodes, x, rowptr, col, y, n_graphs, graph_off, true);
    *loss = (float)tsim::cutnet::loss_grad(params, b, grad);
  });
}

tsim_status tsim_cut_adam_step(float* params, const float* grad, float* m, float* v, int step, float lr) {
  return guard([&] {
    if (!params || !grad || !m || !v) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    tsim::cutnet::adam_step(params, grad, m, v, tsim::cutnet::num_params(), step, lr);
  });
}

tsim_status tsim_cut_train(const char* dataset_path, int epochs, int batch_graphs, float lr, uint64_t seed,
                           float* params, float* loss_per_epoch) {
  return guard([&] {
    if (!dataset_path || !params) tsim::fail(TSIM_ERR_ARG, "NULL argument");
    tsim::cutnet::Batch b = tsim::cutnet::read_dataset(dataset_path);
    tsim::cutnet::train(b, epochs, batch_graphs, lr, seed, params, loss_per_epoch);
  });
}

tsim_status tsim_cut_model_set(const float* params) {
  return guard([&] { tsim::cutnet::set_model(params); });
}

tsim_status tsim_cut_evaluate(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget, double* out) {
  return guard([&] { tsim::cutnet::evaluate_policy(seed, n_graphs, t_min, t_max, budget, out); });
}

tsim_status tsim_cut_policy_stats(uint64_t out[4]) {
  return guard([&] {
    if (!out) tsim::fail(TSIM_ERR_ARG, "NULL out");
    for (int i = 0; i < 4; ++i) out[i] = tsim::g_cut_stats[i].load();
  });
}

}  // extern "C"
