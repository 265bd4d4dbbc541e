// Shard-task scheduler for GPU instances that may leave (Sec. IV "Cloud Instance
// Task Scheduler", "Spot instance cost analysis").  Host code only.
//
//  decide   : one scheduling decision.  Pending tasks are taken longest estimate
//             first (ties: smaller task id).  Availability policy: only idle
//             instances receive a task.  Time-based policy: an instance whose end
//             is announced receives a task only if its remaining time covers the
//             task's estimate; among the instances that can take a task, the one
//             with the least remaining time is chosen (unannounced ends count as
//             unbounded), ties to the smaller instance id.  A task that fits no
//             instance stays pending and smaller tasks are tried next, so an
//             instance about to leave gets the largest task that still fits, or
//             nothing.  Without the time-based policy a task goes to the idle
//             instance of smallest id.
//  simulate : discrete events over instances with start and end times and tasks
//             with estimated and actual durations; a task running when its
//             instance ends is lost and returns to the pending list (reallocation).
//             At one instant, completions come first, then ends, then starts, then
//             one decision.  GPU active time = time instances spend running tasks,
//             lost runs included; cost = makespan x CPU price + GPU active time x
//             GPU price (task durations include their data transfers).
//  estimate : least-squares fit of build time against shard size on timed samples
//             (the paper: time linear in size for one algorithm and machine), or
//             against size^2 (an exact kNN graph costs n^2 d).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/ann.h"

namespace {

struct Pending {
    int id;
    double est;
};

void decide_impl(double now, const std::vector<Pending>& pending, const std::vector<int>& idle,
                 const double* idle_end, int policy, std::vector<int>& task_of_idle) {
    std::vector<Pending> order(pending);
    std::sort(order.begin(), order.end(), [](const Pending& a, const Pending& b) {
        if (a.est != b.est) return a.est > b.est;
        return a.id < b.id;
    });
    task_of_idle.assign(idle.size(), -1);
    for (const Pending& t : order) {
        int best = -1;
        double best_rem = 0.0;
        for (size_t j = 0; j < idle.size(); ++j) {
            if (task_of_idle[j] >= 0) continue;
            if (!(policy & ANN_SCHED_TIME)) {
                if (best < 0 || idle[j] < idle[best]) best = (int)j;
                continue;
            }
            const double rem = idle_end[j] - now;  // +inf when not announced
            if (rem < t.est) continue;
            if (best < 0 || rem < best_rem || (rem == best_rem && idle[j] < idle[best])) {
                best = (int)j;
                best_rem = rem;
            }
        }
        if (best >= 0) task_of_idle[best] = t.id;
    }
}

}  // namespace

extern "C" {

int ann_sched_decide(double now, int n_pending, const int* pending_ids, const double* pending_est,
                     int n_idle, const int* idle_ids, const double* idle_end, int policy,
                     int* task_of_idle) {
    if (n_pending < 0 || n_idle < 0 || (policy & ~ANN_SCHED_TIME)) return ANN_ERR_INVALID_ARG;
    if ((n_pending && (!pending_ids || !pending_est)) ||
        (n_idle && (!idle_ids || !idle_end || !task_of_idle)))
        return ANN_ERR_INVALID_ARG;
    std::vector<Pending> p(n_pending);
    for (int i = 0; i < n_pending; ++i) p[i] = {pending_ids[i], pending_est[i]};
    std::vector<int> idle(idle_ids, idle_ids + n_idle);
    std::vector<int> out;
    decide_impl(now, p, idle, idle_end, policy, out);
    for (int j = 0; j < n_idle; ++j) task_of_idle[j] = out[j];
    return ANN_OK;
}

int ann_sched_simulate(int n_tasks, const double* est, const double* actual, int n_inst,
                       const double* inst_start, const double* inst_end, const int* inst_notice,
                       int policy, double cpu_price, double gpu_price, int* task_inst,
                       double* task_start, double* task_end, int* task_tries,
                       double* summary) {
    if (n_tasks < 0 || n_inst < 0 || (policy & ~ANN_SCHED_TIME)) return ANN_ERR_INVALID_ARG;
    if (n_tasks && (!est || !task_inst || !task_start || !task_end || !task_tries))
        return ANN_ERR_INVALID_ARG;
    if (n_inst && (!inst_start || !inst_end)) return ANN_ERR_INVALID_ARG;
    if (!summary) return ANN_ERR_INVALID_ARG;
    for (int i = 0; i < n_tasks; ++i)
        if (!(est[i] >= 0.0) || (actual && !(actual[i] >= 0.0))) return ANN_ERR_INVALID_ARG;
    for (int j = 0; j < n_inst; ++j)
        if (!(inst_start[j] >= 0.0) || !(inst_end[j] >= inst_start[j])) return ANN_ERR_INVALID_ARG;
    std::vector<int> state(n_tasks, 0);  // 0 pending, 1 running, 2 done
    std::vector<int> run_task(n_inst, -1);
    std::vector<double> run_end(n_inst, 0.0), run_begin(n_inst, 0.0);
    std::vector<char> gone(n_inst, 0);
    for (int i = 0; i < n_tasks; ++i) {
        task_inst[i] = -1;
        task_start[i] = task_end[i] = NAN;
        task_tries[i] = 0;
    }
    double now = 0.0, busy = 0.0, lost = 0.0, makespan = 0.0;
    int realloc = 0, done = 0;
    for (int guard = 0; guard < 4 * (n_tasks + 1) * (n_inst + 1) + 16; ++guard) {
        // completions, then ends, at `now`
        for (int j = 0; j < n_inst; ++j) {
            if (run_task[j] >= 0 && run_end[j] <= now) {
                const int t = run_task[j];
                state[t] = 2;
                task_inst[t] = j;
                task_end[t] = run_end[j];
                busy += run_end[j] - run_begin[j];
                makespan = std::max(makespan, run_end[j]);
                run_task[j] = -1;
                ++done;
            }
        }
        for (int j = 0; j < n_inst; ++j) {
            if (gone[j] || inst_end[j] > now) continue;
            gone[j] = 1;
            if (run_task[j] >= 0) {  // lost: back to the pending list
                const int t = run_task[j];
                state[t] = 0;
                busy += now - run_begin[j];
                lost += now - run_begin[j];
                ++realloc;
                run_task[j] = -1;
            }
        }
        // one decision over the idle instances that are up
        std::vector<Pending> pend;
        for (int i = 0; i < n_tasks; ++i)
            if (state[i] == 0) pend.push_back({i, est[i]});
        std::vector<int> idle;
        std::vector<double> iend;
        for (int j = 0; j < n_inst; ++j)
            if (!gone[j] && inst_start[j] <= now && run_task[j] < 0) {
                idle.push_back(j);
                iend.push_back((inst_notice && inst_notice[j]) ? inst_end[j] : INFINITY);
            }
        if (!pend.empty() && !idle.empty()) {
            std::vector<int> pick;
            decide_impl(now, pend, idle, iend.data(), policy, pick);
            for (size_t q = 0; q < idle.size(); ++q) {
                const int t = pick[q];
                if (t < 0) continue;
                const int j = idle[q];
                state[t] = 1;
                run_task[j] = t;
                run_begin[j] = now;
                run_end[j] = now + (actual ? actual[t] : est[t]);
                if (task_tries[t] == 0) task_start[t] = now;
                ++task_tries[t];
            }
        }
        if (done == n_tasks) break;
        // next event
        double next = INFINITY;
        for (int j = 0; j < n_inst; ++j) {
            if (gone[j]) continue;
            if (run_task[j] >= 0) next = std::min(next, run_end[j]);
            if (inst_start[j] > now) next = std::min(next, inst_start[j]);
            if (inst_start[j] <= now) next = std::min(next, inst_end[j]);
        }
        if (!(next < INFINITY)) break;  // nothing more can happen
        now = next;
    }
    summary[0] = makespan;
    summary[1] = busy;
    summary[2] = lost;
    summary[3] = (double)realloc;
    summary[4] = (double)(n_tasks - done);
    summary[5] = makespan * cpu_price + busy * gpu_price;
    return done == n_tasks ? ANN_OK : ANN_ERR_UNSUPPORTED;
}

int ann_sched_estimate(int n_samples, const double* sample_size, const double* sample_time,
                       int model, int n_tasks, const double* task_size, double* est_out) {
    if (n_samples < 2 || (model != 0 && model != 1) || n_tasks < 0) return ANN_ERR_INVALID_ARG;
    if (!sample_size || !sample_time || (n_tasks && (!task_size || !est_out)))
        return ANN_ERR_INVALID_ARG;
    // least squares of t = a + b f(size), f(s) = s (model 0) or s^2 (model 1)
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int i = 0; i < n_samples; ++i) {
        const double f = model ? sample_size[i] * sample_size[i] : sample_size[i];
        sx += f;
        sy += sample_time[i];
        sxx += f * f;
        sxy += f * sample_time[i];
    }
    const double n = (double)n_samples, den = n * sxx - sx * sx;
    if (!(den != 0.0)) return ANN_ERR_INVALID_ARG;  // all sample sizes equal
    const double b = (n * sxy - sx * sy) / den, a = (sy - b * sx) / n;
    for (int i = 0; i < n_tasks; ++i) {
        const double f = model ? task_size[i] * task_size[i] : task_size[i];
        est_out[i] = a + b * f;
    }
    return ANN_OK;
}

}  // extern "C"
