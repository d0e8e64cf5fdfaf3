// Autotuner of batched ensembles: picks, from timed trials on the caller's own
// systems, each system's leaf size and the batch's launch knobs, and keeps
// the choices in a table that can be cached in a JSON file.
//
// Leaf size, per (size bucket floor(log2 N), profile class, theta, order,
// form): the trial system is the group's system whose size is nearest the
// group's median; every candidate in {8, 16, 32, 64} runs build + gravity on
// it in a scratch context (after one warm-up run that sizes its buffers) and
// the fastest (best of two runs, CUDA events) wins.
//
// Launch knobs, per (total-size bucket, log2 systems, theta, order, form):
// walk schedule {per depth, queue of nodes, queue of sibling pairs} x
// near-field blocks per SM
// {all that fit, one fewer} x neighbour-list chunk {128, 256, 512}, each timed
// on a gravity call of the whole batch.
//
// Profile class: the ratio of the rms to the mean distance from the system's
// centre of mass (1.03 for a homogeneous sphere, about 1.45 for a Plummer
// sphere), cut at 1.1, 1.25 and 1.6 into classes 0 to 3.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "sfmm_internal.cuh"

namespace {

constexpr int TUNE_NT = 256;
constexpr int TUNE_LEAVES[4] = {8, 16, 32, 64};

// One block per system: centre of mass, then the mass-weighted mean and rms
// distance from it.  out[2 s] = mean distance, out[2 s + 1] = rms distance.
__global__ void k_sys_profile(const int64_t* __restrict__ off, const double* __restrict__ pos,
                              const double* __restrict__ mass, double* __restrict__ out) {
  __shared__ double sh[4][TUNE_NT];
  const int s = blockIdx.x;
  const int64_t lo = off[s], hi = off[s + 1];
  double a[4] = {0, 0, 0, 0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += TUNE_NT) {
    const double m = mass[i];
    a[0] += m;
    a[1] += m * pos[3 * i];
    a[2] += m * pos[3 * i + 1];
    a[3] += m * pos[3 * i + 2];
  }
  for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int w = TUNE_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  const double M = sh[0][0];
  const double cx = sh[1][0] / M, cy = sh[2][0] / M, cz = sh[3][0] / M;
  __syncthreads();
  double b[2] = {0, 0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += TUNE_NT) {
    const double m = mass[i];
    const double dx = pos[3 * i] - cx, dy = pos[3 * i + 1] - cy, dz = pos[3 * i + 2] - cz;
    const double r2 = dx * dx + dy * dy + dz * dz;
    b[0] += m * sqrt(r2);
    b[1] += m * r2;
  }
  sh[0][threadIdx.x] = b[0];
  sh[1][threadIdx.x] = b[1];
  __syncthreads();
  for (int w = TUNE_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 2; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * s] = sh[0][0] / M;
    out[2 * s + 1] = sqrt(sh[1][0] / M);
  }
}

int profile_class(double mean, double rms) {
  if (!(mean > 0.0)) return 0;
  const double q = rms / mean;
  return q < 1.1 ? 0 : q < 1.25 ? 1 : q < 1.6 ? 2 : 3;
}

int size_bucket(int64_t n) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << (b + 1)) <= n) ++b;
  return b;
}

const char* form_name(int precision) { return precision == SFMM_FP32 ? "fp32" : "fp64"; }

std::string leaf_key(int bucket, int cls, double theta, int order, int precision) {
  char k[96];
  snprintf(k, sizeof k, "b%d|c%d|t%.3f|p%d|%s", bucket, cls, theta, order, form_name(precision));
  return k;
}

std::string knob_key(int64_t ntot, int nsys, double theta, int order, int precision) {
  char k[96];
  snprintf(k, sizeof k, "N%d|S%d|t%.3f|p%d|%s", size_bucket(ntot), size_bucket(nsys), theta, order,
           form_name(precision));
  return k;
}

float event_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return -1.f;
  }
  return ms;
}

}  // namespace

struct sfmm_tune_table {
  struct Leaf {
    int leaf = 16;
    int64_t trial_n = 0;
    double ms[4] = {0, 0, 0, 0};
  };
  struct Knobs {
    int schedule = 0, p2p_blocks = 0, p2p_chunk = SFMM_P2P_CHUNK_DEFAULT;
    double ms = 0.0;
  };
  std::map<std::string, Leaf> leaf;
  std::map<std::string, Knobs> knobs;
  std::string path;  // cache file ("" = none)
};

namespace sfmm {

void tune_table_free(sfmm_ctx* c) {
  delete c->tune;
  c->tune = nullptr;
}

static sfmm_tune_table* table(sfmm_ctx* c) {
  if (!c->tune) c->tune = new sfmm_tune_table();
  return c->tune;
}

// --- JSON cache: one entry per line, written and read by this file only ----

static int save_table(sfmm_ctx* c) {
  sfmm_tune_table* t = table(c);
  if (t->path.empty()) return SFMM_OK;
  const std::string tmp = t->path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return set_error(c, SFMM_EINVAL, "autotune cache: cannot write the file");
  fprintf(f, "{\n \"leaf\": [\n");
  size_t k = 0;
  for (const auto& e : t->leaf)
    fprintf(f, "  {\"key\": \"%s\", \"leaf_size\": %d, \"trial_n\": %lld, \"ms\": [%.6g, %.6g, %.6g, %.6g]}%s\n",
            e.first.c_str(), e.second.leaf, (long long)e.second.trial_n, e.second.ms[0], e.second.ms[1],
            e.second.ms[2], e.second.ms[3], ++k < t->leaf.size() ? "," : "");
  fprintf(f, " ],\n \"knobs\": [\n");
  k = 0;
  for (const auto& e : t->knobs)
    fprintf(f, "  {\"key\": \"%s\", \"schedule\": %d, \"p2p_blocks\": %d, \"p2p_chunk\": %d, \"ms\": %.6g}%s\n",
            e.first.c_str(), e.second.schedule, e.second.p2p_blocks, e.second.p2p_chunk, e.second.ms,
            ++k < t->knobs.size() ? "," : "");
  fprintf(f, " ]\n}\n");
  const bool ok = fclose(f) == 0 && rename(tmp.c_str(), t->path.c_str()) == 0;
  return ok ? SFMM_OK : set_error(c, SFMM_EINVAL, "autotune cache: cannot write the file");
}

static bool field_int(const char* line, const char* name, long long* v) {
  const char* p = strstr(line, name);
  return p && sscanf(p + strlen(name), " : %lld", v) == 1;
}

static int load_table(sfmm_ctx* c) {
  sfmm_tune_table* t = table(c);
  FILE* f = fopen(t->path.c_str(), "r");
  if (!f) return SFMM_OK;  // no cache yet
  char line[512];
  int section = 0;
  while (fgets(line, sizeof line, f)) {
    if (strstr(line, "\"leaf\":")) section = 1;
    if (strstr(line, "\"knobs\":")) section = 2;
    const char* kp = strstr(line, "\"key\": \"");
    if (!kp) continue;
    kp += 8;
    const char* ke = strchr(kp, '"');
    if (!ke) continue;
    const std::string key(kp, ke - kp);
    long long a = 0, b = 0, d = 0;
    if (section == 1 && field_int(line, "\"leaf_size\"", &a) && a >= 1 && a <= 64) {
      sfmm_tune_table::Leaf e;
      e.leaf = (int)a;
      if (field_int(line, "\"trial_n\"", &b)) e.trial_n = b;
      const char* mp = strstr(line, "\"ms\": [");
      if (mp) sscanf(mp + 7, "%lf , %lf , %lf , %lf", &e.ms[0], &e.ms[1], &e.ms[2], &e.ms[3]);
      t->leaf[key] = e;
    } else if (section == 2 && field_int(line, "\"schedule\"", &a) && field_int(line, "\"p2p_blocks\"", &b) &&
               field_int(line, "\"p2p_chunk\"", &d) && a >= 0 && a <= 3 && b >= 0 && b <= 64 && d >= 32 &&
               d <= 65536) {
      sfmm_tune_table::Knobs e;
      e.schedule = (int)a;
      e.p2p_blocks = (int)b;
      e.p2p_chunk = (int)d;
      t->knobs[key] = e;
    }
  }
  fclose(f);
  return SFMM_OK;
}

// --- trials ------------------------------------------------------------------

// Profile class of every system (one launch, one synchronisation).
static int system_classes(sfmm_ctx* c, int nsys, const int64_t* offsets, const double* pos, const double* mass,
                          std::vector<int>& cls) {
  DevBuf off, out;
  int rc;
  if ((rc = off.ensure(sizeof(int64_t) * (nsys + 1))) || (rc = out.ensure(sizeof(double) * 2 * nsys))) {
    off.release();
    out.release();
    return rc;
  }
  std::vector<double> h(2 * (size_t)nsys);
  cudaError_t e = cudaMemcpyAsync(off.p, offsets, sizeof(int64_t) * (nsys + 1), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    k_sys_profile<<<nsys, TUNE_NT, 0, c->stream>>>(off.as<int64_t>(), pos, mass, out.as<double>());
    ++c->nlaunch;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), out.p, sizeof(double) * 2 * nsys, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  off.release();
  out.release();
  if (e != cudaSuccess) return set_error(c, SFMM_ECUDA, cudaGetErrorString(e));
  cls.resize(nsys);
  for (int s = 0; s < nsys; ++s) cls[s] = profile_class(h[2 * s], h[2 * s + 1]);
  return SFMM_OK;
}

// Timed build + gravity of one system per candidate leaf size, in a scratch
// context with the caller's options.
static int time_leaf_sizes(sfmm_ctx* c, int64_t n, const double* pos, const double* mass, const double* h,
                           double theta, int order, sfmm_tune_table::Leaf* best) {
  sfmm_ctx* t = nullptr;
  int rc = sfmm_create(&t, c->device, c->precision, c->stream);
  if (rc) return set_error(c, rc, "autotune: scratch context");
  t->G = c->G;
  t->walk_mode = c->walk_mode;
  t->schedule = c->schedule;
  t->p2p_chunk = c->p2p_chunk;
  t->p2p_blocks = c->p2p_blocks;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((rc = t->out_acc.ensure(sizeof(double) * 3 * (size_t)n)) || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    if (!rc) rc = SFMM_ECUDA;
  }
  double best_ms = 1e300;
  for (int k = 0; rc == SFMM_OK && k < 4; ++k) {
    const int leaf = TUNE_LEAVES[k];
    double ms_k = 1e300;
    for (int rep = 0; rc == SFMM_OK && rep < 3; ++rep) {  // first run sizes the buffers
      cudaEventRecord(e0, t->stream);
      if ((rc = sfmm_build(t, n, pos, mass, h, leaf)) ||
          (rc = sfmm_gravity(t, theta, order, t->out_acc.as<double>(), nullptr)))
        break;
      cudaEventRecord(e1, t->stream);
      const float ms = event_ms(e0, e1);
      if (ms < 0.f) rc = SFMM_ECUDA;
      if (rep > 0) ms_k = std::min(ms_k, (double)ms);
    }
    best->ms[k] = ms_k;
    if (rc == SFMM_OK && ms_k < best_ms) {
      best_ms = ms_k;
      best->leaf = leaf;
    }
  }
  best->trial_n = n;
  if (rc) c->last_error = std::string("autotune trial: ") + t->last_error;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  sfmm_destroy(t);
  return rc;
}

// Leaf sizes of every system from the table, running the trials of groups
// that have no entry yet.
int tuned_leaf_sizes(sfmm_ctx* c, int nsys, const int64_t* offsets, const double* pos, const double* mass,
                     const double* h, double theta, int order, std::vector<int>& lsz) {
  sfmm_tune_table* t = table(c);
  std::vector<int> cls;
  int rc = system_classes(c, nsys, offsets, pos, mass, cls);
  if (rc) return rc;
  std::map<std::string, std::vector<int>> groups;
  std::vector<std::string> key(nsys);
  for (int s = 0; s < nsys; ++s) {
    key[s] = leaf_key(size_bucket(offsets[s + 1] - offsets[s]), cls[s], theta, order, c->precision);
    groups[key[s]].push_back(s);
  }
  bool added = false;
  for (auto& g : groups) {
    if (t->leaf.count(g.first)) continue;
    std::vector<int>& v = g.second;
    std::vector<int64_t> sizes;
    for (int s : v) sizes.push_back(offsets[s + 1] - offsets[s]);
    std::vector<int64_t> sorted = sizes;
    std::nth_element(sorted.begin(), sorted.begin() + sorted.size() / 2, sorted.end());
    const int64_t med = sorted[sorted.size() / 2];
    int rep = v[0];
    for (size_t k = 0; k < v.size(); ++k)
      if (std::llabs(sizes[k] - med) < std::llabs(offsets[rep + 1] - offsets[rep] - med)) rep = v[k];
    const int64_t o = offsets[rep], n = offsets[rep + 1] - offsets[rep];
    sfmm_tune_table::Leaf e;
    if ((rc = time_leaf_sizes(c, n, pos + 3 * o, mass + o, h + o, theta, order, &e))) return rc;
    t->leaf[g.first] = e;
    added = true;
  }
  lsz.resize(nsys);
  for (int s = 0; s < nsys; ++s) lsz[s] = t->leaf[key[s]].leaf;
  return added ? save_table(c) : SFMM_OK;
}

// Launch knobs of the built batch from the table, running the trials when the
// batch has no entry yet (acc: device scratch of the batch's size).
int tuned_knobs(sfmm_ctx* c, double theta, int order, double* acc, bool run_trials) {
  sfmm_tune_table* t = table(c);
  const std::string k = knob_key(c->n, c->nsys, theta, order, c->precision);
  auto it = t->knobs.find(k);
  if (it == t->knobs.end()) {
    if (!run_trials) return SFMM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      cudaGetLastError();
      return SFMM_ECUDA;
    }
    sfmm_tune_table::Knobs best;
    best.ms = 1e300;
    int rc = SFMM_OK;
    const int schedules[3] = {1, 2, 3};
    const int chunks[3] = {128, 256, 512};
    const int fit = p2p_blocks_fit(c);  // near-field blocks per SM that fit
    const int nb = fit > 1 ? 2 : 1;     // all that fit, and one fewer
    for (int si = 0; rc == SFMM_OK && si < 3; ++si)
      for (int bi = 0; rc == SFMM_OK && bi < nb; ++bi)
        for (int ci = 0; rc == SFMM_OK && ci < 3; ++ci) {
          c->schedule = schedules[si];
          c->p2p_blocks = bi ? fit - 1 : 0;
          c->p2p_chunk = chunks[ci];
          double ms_k = 1e300;
          for (int rep = 0; rc == SFMM_OK && rep < 3; ++rep) {  // first run regrows buffers
            cudaEventRecord(e0, c->stream);
            if ((rc = sfmm_gravity(c, theta, order, acc, nullptr))) break;
            cudaEventRecord(e1, c->stream);
            const float ms = event_ms(e0, e1);
            if (ms < 0.f) rc = SFMM_ECUDA;
            if (rep > 0) ms_k = std::min(ms_k, (double)ms);
          }
          if (rc == SFMM_OK && ms_k < best.ms) {
            best.ms = ms_k;
            best.schedule = c->schedule;
            best.p2p_blocks = c->p2p_blocks;
            best.p2p_chunk = c->p2p_chunk;
          }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    t->knobs[k] = best;
    if ((rc = save_table(c))) return rc;
    it = t->knobs.find(k);
  }
  c->schedule = it->second.schedule;
  c->p2p_blocks = it->second.p2p_blocks;
  c->p2p_chunk = it->second.p2p_chunk;
  return SFMM_OK;
}

int tune_set_cache(sfmm_ctx* c, const char* path) {
  sfmm_tune_table* t = table(c);
  t->path = path ? path : "";
  if (t->path.empty()) return SFMM_OK;
  return load_table(c);
}

}  // namespace sfmm
