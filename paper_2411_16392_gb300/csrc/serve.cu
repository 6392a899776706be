// Serving loop: resident scenes, bounded FIFO queue, memory-budget admission, worker
// slots with their own rendering context and stream (continuous batching: requests are
// admitted as slots and budget free up, the kernels of the slots in flight overlap, and a
// single-slot server's free slot takes the queue's head together with the other queued
// small views of the same scene and renders them in shared launches, render_forward_batch;
// see batch_pays).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/qgs_serve.h"
#include "qgs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct SceneDev {
  int64_t n = 0;
  float *mean = nullptr, *quat = nullptr, *scale = nullptr, *curv = nullptr, *opacity = nullptr;
  uint16_t* sh = nullptr;
  double inst_per_pixel = 64.0;  // running estimate of tile instances per pixel
};

struct Request {
  uint64_t ticket = 0;
  int32_t scene = 0;
  SceneDev scn;  // copy of the scene's pointers taken at submission
  qgs_camera cam{};
  Clock::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done
  qgs_status status = QGS_OK;
  int64_t est_bytes = 0;
  float* result = nullptr;       // 8 planes of W*H floats (device, or host in fake mode)
  bool result_on_host = false;
  bool want_bwd = false;         // forward + backward request
  float* grad_in = nullptr;      // upstream gradient planes, 8 x W*H (device; null: zero)
  float* grads = nullptr;        // parameter gradients, 60 floats per primitive (device or host)
};

// Parameter-gradient layout of a backward request's result: mean 3n, quat 4n, scale 2n,
// curv 2n, opacity n, sh 48n floats (the qgs_scene_grad arrays, back to back).
constexpr int kGradFloats = 60;
inline qgs_scene_grad grad_view(float* g, int64_t n) {
  return qgs_scene_grad{g, g + 3 * n, g + 7 * n, g + 9 * n, g + 11 * n, g + 12 * n};
}

struct Slot {
  qgs_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::thread th;
};

// Shared launches save a view its own launches and host round trip (a fixed cost per frame)
// but share none of its work: every view preprocesses, sorts and composites its own entries,
// and the joint sorts cost a little more per view than separate ones. A server with several
// slots already hides each frame's fixed cost behind the other slots' kernels, and there
// concurrent single renders measured faster than batches at every scene size and frame size
// tried (0.2M and 1M quadrics at 256^2, 512x384 and 1024x768: 4 slots 1.0-1.3x the frames/s
// of 4 slots batching up to 8 views). With one slot nothing hides it, and batches of up to 8
// small views measured 1.2-2.1x the frames/s of one-at-a-time renders at 256^2 and 512x384
// (no gain at 1024x768). So only a single-slot server batches, and only frames up to 512x384.
constexpr int64_t kBatchMaxPixels = 512 * 384;
inline bool batch_pays(int n_slots, const qgs_camera& c) {
  return n_slots == 1 && (int64_t)c.W * c.H <= kBatchMaxPixels;
}

int64_t request_bytes(const SceneDev& s, const qgs_camera& c, bool bwd) {
  const double P = (double)c.W * c.H;
  const double inst = s.inst_per_pixel * P;
  // projected state + per-primitive keys/indices/offsets, tile-test bounds and mask
  // offsets, instance ping-pong buffers, radix histogram, residue, the 8 result planes and
  // the tile masks; a backward adds the per-primitive gradient records, the parameter
  // gradients and the upstream planes
  double b = s.n * 252.0 + inst * 16.0 + inst / 16.0 + P * 8.0 + P * 32.0 + 16.0 * (1 << 20);
  if (bwd) b += s.n * (80.0 + 4.0 * kGradFloats) + P * 32.0;
  return (int64_t)b + (1 << 20);
}

}  // namespace

namespace qgs {
// defined in api.cu: instance count of the context's last forward
int64_t last_instance_count(const qgs_ctx* ctx);
}  // namespace qgs

struct qgs_server {
  int device = 0;
  bool fake = false;
  double fake_us_per_mpix = 0;
  int64_t budget = 0;
  int queue_cap = 0;
  int max_batch = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::deque<SceneDev> scenes;  // references stay valid as scenes are added
  std::vector<Slot> slots;
  cudaStream_t copy_stream = nullptr;
  uint64_t next_ticket = 1;
  int64_t reserved = 0;
  int running = 0;
  bool stop = false;
  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0, rejected = 0, max_in_flight = 0, reserved_peak = 0;
  int64_t batches = 0, max_batch_seen = 0;
  bool have_first = false;
  Clock::time_point t_first, t_last;

  void worker(int slot_index);
  void run_batch(Slot& s, std::vector<Request*>& batch);
};

void qgs_server::run_batch(Slot& s, std::vector<Request*>& batch) {
  if (fake) {
    int64_t P_all = 0;
    for (Request* r : batch) {
      const int64_t P = (int64_t)r->cam.W * r->cam.H;
      P_all += r->want_bwd ? 3 * P : P;  // a backward costs about twice a forward
      r->result = static_cast<float*>(calloc((size_t)P * 8, sizeof(float)));
      r->result_on_host = true;
      r->status = r->result ? QGS_OK : QGS_ENOMEM;
      if (r->want_bwd) {
        r->grads = static_cast<float*>(calloc((size_t)std::max<int64_t>(r->scn.n, 1) * kGradFloats, sizeof(float)));
        if (!r->grads) r->status = QGS_ENOMEM;
      }
    }
    const double us = fake_us_per_mpix * (double)P_all / 1e6;
    std::this_thread::sleep_for(std::chrono::microseconds((int64_t)us));
    return;
  }
  cudaSetDevice(device);
  const SceneDev& sc = batch[0]->scn;
  std::vector<qgs_camera> cams;
  std::vector<qgs_image> outs;
  int64_t P_all = 0;
  qgs_status st = QGS_OK;
  for (Request* r : batch) {
    const int64_t P = (int64_t)r->cam.W * r->cam.H;
    void* buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, sizeof(float) * 8 * (size_t)P, s.stream);
    if (e != cudaSuccess) {
      st = e == cudaErrorMemoryAllocation ? QGS_ENOMEM : QGS_ECUDA;
      break;
    }
    r->result = static_cast<float*>(buf);
    cams.push_back(r->cam);
    outs.push_back(qgs_image{r->result, r->result + 3 * P, r->result + 4 * P, r->result + 5 * P});
    P_all += P;
  }
  qgs_scene scn{sc.n, sc.mean, sc.quat, sc.scale, sc.curv, sc.opacity, sc.sh};
  if (st == QGS_OK) {
    if (batch.size() == 1)
      st = render_forward(s.ctx, &scn, &cams[0], &outs[0], s.stream);
    else
      st = render_forward_batch(s.ctx, &scn, (int32_t)batch.size(), cams.data(), outs.data(), s.stream);
  }
  if (st == QGS_OK && batch.size() == 1 && batch[0]->want_bwd) {
    // a backward request runs alone: gradients of sum(grad_in . planes) into its buffer
    Request* r = batch[0];
    const int64_t P = (int64_t)r->cam.W * r->cam.H;
    void* g = nullptr;
    cudaError_t e = cudaMallocAsync(&g, sizeof(float) * kGradFloats * (size_t)std::max<int64_t>(sc.n, 1), s.stream);
    if (e != cudaSuccess) {
      st = e == cudaErrorMemoryAllocation ? QGS_ENOMEM : QGS_ECUDA;
    } else {
      r->grads = static_cast<float*>(g);
      if (cudaMemsetAsync(g, 0, sizeof(float) * kGradFloats * (size_t)sc.n, s.stream) != cudaSuccess) st = QGS_ECUDA;
      float* gi = r->grad_in;
      qgs_image gin{gi, gi ? gi + 3 * P : nullptr, gi ? gi + 4 * P : nullptr, gi ? gi + 5 * P : nullptr};
      const qgs_scene_grad gv = grad_view(r->grads, sc.n);
      if (st == QGS_OK) st = render_backward(s.ctx, &scn, &r->cam, &gin, &gv, s.stream);
    }
  }
  if (st == QGS_OK && cudaStreamSynchronize(s.stream) != cudaSuccess) st = QGS_ECUDA;
  if (st == QGS_OK) st = qgs_check_frame(s.ctx);  // the frame's sorts completed their waits
  for (Request* r : batch) r->status = st;
  if (st == QGS_OK) {
    const int64_t inst = qgs::last_instance_count(s.ctx);
    std::lock_guard<std::mutex> lk(mu);
    SceneDev& sd = scenes[batch[0]->scene];
    sd.inst_per_pixel = 0.7 * sd.inst_per_pixel + 0.3 * ((double)inst / (double)std::max<int64_t>(P_all, 1));
  }
}

void qgs_server::worker(int si) {
  Slot& s = slots[si];
  if (!fake) cudaSetDevice(device);
  std::vector<Request*> batch;
  for (;;) {
    int64_t est = 0;
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] {
        if (stop) return true;
        if (queue.empty()) return false;
        // FIFO head is admitted when it fits in the remaining budget (or nothing runs)
        return running == 0 || reserved + queue.front()->est_bytes <= budget;
      });
      if (stop) return;
      Request* head = queue.front();
      queue.pop_front();
      batch.push_back(head);
      est = head->est_bytes;
      // the other queued forward views of the same scene that still fit join the head's
      // launches where sharing them pays (a backward request runs alone; see batch_pays)
      const int n_slots = (int)slots.size();
      for (auto it = queue.begin(); it != queue.end() && !head->want_bwd && (int)batch.size() < max_batch &&
                                    batch_pays(n_slots, head->cam);) {
        Request* r = *it;
        if (!r->want_bwd && r->scene == head->scene && batch_pays(n_slots, r->cam) &&
            reserved + est + r->est_bytes <= budget) {
          batch.push_back(r);
          est += r->est_bytes;
          it = queue.erase(it);
        } else {
          ++it;
        }
      }
      for (Request* r : batch) r->state = 1;
      reserved += est;
      running += (int)batch.size();
      ++batches;
      max_batch_seen = std::max<int64_t>(max_batch_seen, (int64_t)batch.size());
      max_in_flight = std::max<int64_t>(max_in_flight, running);
      reserved_peak = std::max(reserved_peak, reserved);
    }
    run_batch(s, batch);
    {
      std::lock_guard<std::mutex> lk(mu);
      const Clock::time_point now = Clock::now();
      for (Request* r : batch) {
        r->t_done = now;
        r->state = 2;
        ++completed;
        if (r->status != QGS_OK) ++failed;
        lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
      }
      reserved -= est;
      running -= (int)batch.size();
      t_last = now;
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

qgs_status serve_create(qgs_server** out, int32_t device, int64_t hbm_budget_bytes, int32_t max_slots,
                        int32_t max_batch, int32_t queue_capacity, double fake_us_per_mpix) {
  if (!out || max_slots < 1 || max_slots > 64 || max_batch < 1 || max_batch > 1024 || queue_capacity < 1 ||
      hbm_budget_bytes <= 0)
    return QGS_EINVAL;
  *out = nullptr;
  std::unique_ptr<qgs_server> s(new (std::nothrow) qgs_server());
  if (!s) return QGS_ENOMEM;
  s->device = device;
  s->fake = device < 0;
  s->fake_us_per_mpix = fake_us_per_mpix;
  s->budget = hbm_budget_bytes;
  s->queue_cap = queue_capacity;
  s->max_batch = max_batch;
  s->slots.resize(max_slots);
  if (!s->fake) {
    if (cudaSetDevice(device) != cudaSuccess) return QGS_ECUDA;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;  // keep freed result buffers cached in the pool
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    // result copies go to caller memory: a blocking stream, ordered after the caller's
    // work on the legacy default stream (e.g. the initialisation of the destination)
    if (cudaStreamCreate(&s->copy_stream) != cudaSuccess) return QGS_ECUDA;
    for (auto& sl : s->slots) {
      qgs_status st = qgs_create(&sl.ctx, nullptr, device);
      if (st != QGS_OK) {
        for (auto& t : s->slots) {
          if (t.ctx) qgs_destroy(t.ctx);
          if (t.stream) cudaStreamDestroy(t.stream);
        }
        cudaStreamDestroy(s->copy_stream);
        return st;
      }
      if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) return QGS_ECUDA;
      qgs_set_pair_counters(sl.ctx, 0);  // serving reads no per-pair counters
    }
  }
  qgs_server* raw = s.release();
  for (int i = 0; i < max_slots; ++i) raw->slots[i].th = std::thread(&qgs_server::worker, raw, i);
  *out = raw;
  return QGS_OK;
}

void serve_destroy(qgs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& sl : s->slots)
    if (sl.th.joinable()) sl.th.join();
  if (!s->fake) cudaSetDevice(s->device);
  for (auto& kv : s->reqs) {
    Request* r = kv.second.get();
    if (r->result_on_host) {
      free(r->result);
      free(r->grads);
    } else {
      if (r->result) cudaFree(r->result);
      if (r->grads) cudaFree(r->grads);
    }
    if (r->grad_in) cudaFree(r->grad_in);
  }
  for (auto& sl : s->slots) {
    if (sl.ctx) qgs_destroy(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (!s->fake) {
    for (auto& sc : s->scenes) {
      cudaFree(sc.mean); cudaFree(sc.quat); cudaFree(sc.scale); cudaFree(sc.curv); cudaFree(sc.opacity);
      cudaFree(sc.sh);
    }
  }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  delete s;
}

qgs_status serve_load_scene(qgs_server* s, const qgs_scene* sc, int32_t* scene_id) {
  if (!s || !sc || !scene_id || sc->n < 0 || sc->n > (int64_t)0x7FFFFFFF) return QGS_EINVAL;
  SceneDev d;
  d.n = sc->n;
  if (!s->fake && sc->n > 0) {
    if (!sc->mean || !sc->quat || !sc->scale || !sc->curv || !sc->opacity || !sc->sh) return QGS_EINVAL;
    cudaSetDevice(s->device);
    const size_t n = (size_t)sc->n;
    struct Item {
      void** dst;
      const void* src;
      size_t bytes;
    } items[] = {{(void**)&d.mean, sc->mean, 12 * n},  {(void**)&d.quat, sc->quat, 16 * n},
                 {(void**)&d.scale, sc->scale, 8 * n}, {(void**)&d.curv, sc->curv, 8 * n},
                 {(void**)&d.opacity, sc->opacity, 4 * n}, {(void**)&d.sh, sc->sh, 96 * n}};
    for (auto& it : items) {
      if (cudaMalloc(it.dst, it.bytes) != cudaSuccess) {
        for (auto& jt : items)
          if (*jt.dst) cudaFree(*jt.dst);
        return QGS_ENOMEM;
      }
      // a device-to-device cudaMemcpy may return before the copy is done, and the
      // workers' streams do not wait for the default stream: copy on the server's copy
      // stream (ordered after the caller's default-stream work) and wait for it here
      if (cudaMemcpyAsync(*it.dst, it.src, it.bytes, cudaMemcpyDefault, s->copy_stream) != cudaSuccess) {
        cudaStreamSynchronize(s->copy_stream);
        for (auto& jt : items)
          if (*jt.dst) cudaFree(*jt.dst);
        return QGS_ECUDA;
      }
    }
    if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess) {
      for (auto& jt : items)
        if (*jt.dst) cudaFree(*jt.dst);
      return QGS_ECUDA;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->scenes.push_back(d);
  *scene_id = (int32_t)s->scenes.size() - 1;
  return QGS_OK;
}

qgs_status serve_submit(qgs_server* s, int32_t scene_id, const qgs_camera* cam, int32_t want_backward,
                        const qgs_image* grad_out, uint64_t* ticket) {
  if (!s || !cam || !ticket) return QGS_EINVAL;
  if (cam->W <= 0 || cam->H <= 0 || cam->W > 32768 || cam->H > 32768 || !(cam->fx > 0) || !(cam->fy > 0) ||
      !(cam->near_plane > 0))
    return QGS_EINVAL;
  if (grad_out && (grad_out->curvature || grad_out->distortion || grad_out->median_depth)) return QGS_EINVAL;
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return QGS_ENOMEM;
  r->want_bwd = want_backward != 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size()) return QGS_ENOTFOUND;
    r->scn = s->scenes[scene_id];
  }
  const int64_t P = (int64_t)cam->W * cam->H;
  if (r->want_bwd && !s->fake && grad_out &&
      (grad_out->rgb || grad_out->alpha || grad_out->depth || grad_out->normal)) {
    // the upstream planes are copied now, so the caller may reuse its buffers at once
    cudaSetDevice(s->device);
    void* g = nullptr;
    if (cudaMalloc(&g, sizeof(float) * 8 * (size_t)P) != cudaSuccess) return QGS_ENOMEM;
    r->grad_in = static_cast<float*>(g);
    const float* src[4] = {grad_out->rgb, grad_out->alpha, grad_out->depth, grad_out->normal};
    const size_t off[4] = {0, 3 * (size_t)P, 4 * (size_t)P, 5 * (size_t)P};
    const size_t cnt[4] = {3 * (size_t)P, (size_t)P, (size_t)P, 3 * (size_t)P};
    bool ok = true;
    for (int k = 0; k < 4 && ok; ++k) {
      if (src[k])
        ok = cudaMemcpyAsync(r->grad_in + off[k], src[k], sizeof(float) * cnt[k], cudaMemcpyDefault,
                             s->copy_stream) == cudaSuccess;
      else
        ok = cudaMemsetAsync(r->grad_in + off[k], 0, sizeof(float) * cnt[k], s->copy_stream) == cudaSuccess;
    }
    if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess) ok = false;
    if (!ok) {
      cudaFree(r->grad_in);
      return QGS_ECUDA;
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->queue.size() >= s->queue_cap) {
      ++s->rejected;
      if (r->grad_in) cudaFree(r->grad_in);
      return QGS_EBUSY;
    }
    r->est_bytes = request_bytes(r->scn, *cam, r->want_bwd);
    if (r->est_bytes > s->budget) {
      ++s->rejected;
      if (r->grad_in) cudaFree(r->grad_in);
      return QGS_ECAPACITY;
    }
    r->ticket = s->next_ticket++;
    r->scene = scene_id;
    r->cam = *cam;
    r->t_submit = Clock::now();
    if (!s->have_first) {
      s->have_first = true;
      s->t_first = r->t_submit;
    }
    ++s->submitted;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs.emplace(r->ticket, std::move(r));
  }
  s->cv_work.notify_one();
  return QGS_OK;
}

qgs_status serve_wait(qgs_server* s, uint64_t ticket, int32_t timeout_ms, const qgs_image* out,
                      const qgs_scene_grad* grad) {
  if (!s) return QGS_EINVAL;
  if (out && (out->curvature || out->distortion || out->median_depth)) return QGS_EINVAL;  // base planes only
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return QGS_ENOTFOUND;
    r = it->second.get();
    if (grad && !r->want_bwd) return QGS_EINVAL;  // a forward request has no gradients
    auto done = [&] { return r->state == 2; };
    if (timeout_ms < 0) {
      s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
      return QGS_ETIMEDOUT;
    }
  }
  qgs_status st = r->status;
  const size_t P = (size_t)r->cam.W * r->cam.H;
  if (st == QGS_OK && out && r->result) {
    float* planes[4] = {out->rgb, out->alpha, out->depth, out->normal};
    const size_t off[4] = {0, 3 * P, 4 * P, 5 * P};
    const size_t cnt[4] = {3 * P, P, P, 3 * P};
    if (r->result_on_host) {
      for (int k = 0; k < 4; ++k)
        if (planes[k]) {
          if (s->fake)
            memcpy(planes[k], r->result + off[k], sizeof(float) * cnt[k]);
        }
    } else {
      cudaSetDevice(s->device);
      for (int k = 0; k < 4 && st == QGS_OK; ++k)
        if (planes[k] &&
            cudaMemcpyAsync(planes[k], r->result + off[k], sizeof(float) * cnt[k], cudaMemcpyDefault,
                            s->copy_stream) != cudaSuccess)
          st = QGS_ECUDA;
      if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess) st = QGS_ECUDA;
    }
  }
  if (st == QGS_OK && grad && r->grads) {
    const int64_t n = r->scn.n;
    float* dst[6] = {grad->mean, grad->quat, grad->scale, grad->curv, grad->opacity, grad->sh};
    const qgs_scene_grad gv = grad_view(r->grads, n);
    const float* src[6] = {gv.mean, gv.quat, gv.scale, gv.curv, gv.opacity, gv.sh};
    const size_t cnt[6] = {3 * (size_t)n, 4 * (size_t)n, 2 * (size_t)n, 2 * (size_t)n, (size_t)n, 48 * (size_t)n};
    if (r->result_on_host) {
      for (int k = 0; k < 6; ++k)
        if (dst[k] && n > 0) memcpy(dst[k], src[k], sizeof(float) * cnt[k]);
    } else {
      cudaSetDevice(s->device);
      for (int k = 0; k < 6 && st == QGS_OK; ++k)
        if (dst[k] && n > 0 &&
            cudaMemcpyAsync(dst[k], src[k], sizeof(float) * cnt[k], cudaMemcpyDefault, s->copy_stream) != cudaSuccess)
          st = QGS_ECUDA;
      if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess) st = QGS_ECUDA;
    }
  }
  if (r->result_on_host) {
    free(r->result);
    free(r->grads);
  } else {
    cudaSetDevice(s->device);
    if (r->result) cudaFreeAsync(r->result, s->copy_stream);
    if (r->grads) cudaFreeAsync(r->grads, s->copy_stream);
  }
  if (r->grad_in) {
    cudaSetDevice(s->device);
    cudaFree(r->grad_in);
  }
  r->result = nullptr;
  r->grads = nullptr;
  r->grad_in = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  s->reqs.erase(ticket);
  return st;
}

qgs_status serve_stats(qgs_server* s, qgs_serve_stats* out) {
  if (!s || !out) return QGS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->rejected = s->rejected;
  out->max_in_flight = s->max_in_flight;
  out->bytes_budget = s->budget;
  out->bytes_reserved_peak = s->reserved_peak;
  out->batches = s->batches;
  out->max_batch = s->max_batch_seen;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
    const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
    out->frames_per_s = span > 0 ? (double)s->completed / span : 0.0;
  }
  return QGS_OK;
}

qgs_status serve_reset_stats(qgs_server* s) {
  if (!s) return QGS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ms.clear();
  s->submitted = s->completed = s->failed = s->rejected = 0;
  s->batches = s->max_batch_seen = 0;
  s->max_in_flight = s->running;
  s->reserved_peak = s->reserved;
  s->have_first = false;
  return QGS_OK;
}

}  // extern "C"
