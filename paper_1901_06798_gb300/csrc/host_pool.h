// host_pool.h -- persistent host worker threads for the regrid path
// (clustering, level tables).  A regrid runs several short parallel loops; at
// a few microseconds each, spawning and joining 16 threads per loop cost as
// much as the loops themselves.  One pool per process, created on first use and
// never torn down (its idle workers block on a condition variable).
#pragma once
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include <unistd.h>

namespace tsu {

class HostPool {
public:
    // The pool of this process.  A child forked after the pool started has the
    // object but not its threads, so a new pool is made for the child (the
    // parent's copy is left as it is).
    static HostPool &get()
    {
        static std::mutex mk;
        static HostPool *p = nullptr;
        static pid_t owner = 0;
        std::lock_guard<std::mutex> lk(mk);
        if (!p || owner != getpid()) {
            p = new HostPool(std::max(1, std::min(16, (int)std::thread::hardware_concurrency())));
            owner = getpid();
        }
        return *p;
    }
    int size() const { return nthreads_; }

    // f(k) for every k in [0, n), on the calling thread and the workers;
    // returns when all are done.  One loop at a time: callers serialise.
    //
    // A worker joins a loop only after taking the job under the mutex (active_
    // counts those in it), and a new loop starts only once no worker is still
    // inside the last one, so job_, njobs_ and the index counter are never
    // read across two loops.
    void run(int n, const std::function<void(int)> &f)
    {
        if (n <= 0) return;
        if (n == 1 || nthreads_ == 1) {
            for (int k = 0; k < n; k++) f(k);
            return;
        }
        std::lock_guard<std::mutex> one(run_mu_);
        {
            std::unique_lock<std::mutex> lk(mu_);
            idle_cv_.wait(lk, [&] { return active_ == 0; });
            job_ = &f;
            njobs_ = n;
            next_.store(0);
            pending_ = n;
            gen_++;
        }
        cv_.notify_all();
        work();
        std::unique_lock<std::mutex> lk(mu_);
        idle_cv_.wait(lk, [&] { return pending_ == 0 && active_ == 0; });
        job_ = nullptr;
    }

private:
    explicit HostPool(int n) : nthreads_(n)
    {
        for (int k = 1; k < n; k++) {
            std::thread t([this] { loop(); });
            t.detach();
        }
    }
    void work()
    {
        int done = 0;
        for (;;) {
            const int k = next_.fetch_add(1);
            if (k >= njobs_) break;
            (*job_)(k);
            done++;
        }
        if (done) {
            std::lock_guard<std::mutex> lk(mu_);
            pending_ -= done;
        }
        idle_cv_.notify_all();
    }
    void loop()
    {
        long seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                active_++;
            }
            work();
            {
                std::lock_guard<std::mutex> lk(mu_);
                active_--;
            }
            idle_cv_.notify_all();
        }
    }

    const int nthreads_;
    std::mutex run_mu_, mu_;
    std::condition_variable cv_, idle_cv_;
    const std::function<void(int)> *job_ = nullptr;
    int njobs_ = 0;
    std::atomic<int> next_{0};
    int pending_ = 0;
    int active_ = 0;   // workers inside the current loop
    long gen_ = 0;
};

}  // namespace tsu
