// Lockstep rounds of independent workers (host side, no CUDA): each worker,
// when it needs a round, arrives with a request and waits; the last of the
// workers still taking part to arrive runs the round for every waiting
// request (under the lock) and wakes them.  A worker that stops taking part
// leaves; if everyone left is waiting, the leaver runs their round.  So a
// round never waits for a worker that will not arrive, and every arrival is
// served by exactly one round.  The batched solve runs its Arnoldi steps this
// way (one graph launch per round); the logic is tested on the host.
#pragma once
#include <condition_variable>
#include <mutex>
#include <utility>
#include <vector>

namespace prd {

template <typename Req>
class Lockstep {
 public:
  explicit Lockstep(int live) : live_(live) {}

  // Join the current round with request r.  launch(const std::vector<Req>&)
  // returns an int status that every worker of the round receives.
  template <typename Launch>
  int arrive(const Req& r, Launch&& launch) {
    std::unique_lock<std::mutex> lk(mu_);
    const long long g = gen_;
    req_.push_back(r);
    if ((int)req_.size() == live_) {
      run(launch);
      return status_;
    }
    cv_.wait(lk, [&] { return gen_ != g; });
    return status_;
  }

  // Stop taking part; if every worker left is waiting, run their round.
  template <typename Launch>
  void leave(Launch&& launch) {
    std::unique_lock<std::mutex> lk(mu_);
    --live_;
    if (!req_.empty() && (int)req_.size() == live_) run(launch);
  }

  long long rounds() const { return gen_; }

 private:
  template <typename Launch>
  void run(Launch& launch) {
    status_ = launch(static_cast<const std::vector<Req>&>(req_));
    req_.clear();
    ++gen_;
    cv_.notify_all();
  }

  std::mutex mu_;
  std::condition_variable cv_;
  int live_;
  long long gen_ = 0;
  std::vector<Req> req_;
  int status_ = 0;
};

}  // namespace prd
