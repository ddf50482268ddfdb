"""The reference arm of bench.py (the oracle timed on the host cores) keeps the JSON-line
contract on CPU: one line with the metric, unit and config of the GPU arm, impl =
"reference", a cpu_baseline describing the run and an e2e object with zero transfers;
under torch.distributed.run with two ranks only rank 0 prints, on all the host cores
the process may use, and both exit 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--steps", "2", "--warmup", "1", "--workload", "plain_n1e3"]


def _json_lines(out):
    return [json.loads(line) for line in out.splitlines() if line.startswith("{")]


def _check_line(d, n_gpus):
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == n_gpus and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == "plain_n1e3" and d["config"]["N"] == 1000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


def test_reference_arm_under_torchrun_prints_once():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2", *ARGS]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 2)
    # the launcher's OMP_NUM_THREADS=1 does not limit the oracle: it uses the host's cores
    assert lines[0]["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))


def test_reference_arm_sizes_each_step_for_the_requested_step_count():
    """The reference arm's sample per step: at least one wave vector per core (the
    oracle's structure factors run one wave vector per thread), and a prefix of the
    particles sized so that steps x sample time stays near two minutes, at most 2 s a step."""
    import bench
    N, P, rate = 1000000, 500, 2.0e6  # (particle, wave vector) pairs per second
    for steps, cores in ((20, 16), (300, 16), (1000, 8), (5, 72)):
        n_s, p_s = bench._reference_sample(N, P, cores, 4, rate, steps, 3)
        assert p_s == min(P, max(4, cores)) and n_s % 2 == 0 and 2 <= n_s <= N
        t_step = n_s * p_s / rate
        assert t_step <= 2.0 + 1e-9 and steps * t_step <= 121.0, (steps, cores, t_step)
    # a tiny workload is evaluated whole
    assert bench._reference_sample(1000, 100, 16, 4, rate, 2, 1) == (1000, 16)


def test_oracle_workload_timings_report_both_sums():
    """bench.py's timings of the explicit-image oracle at the small configurations: the
    random-batch estimator and the full k-sum, each a scaled sample with its size named."""
    import bench
    out = bench.oracle_workloads(target_s=0.05)
    assert set(out) == {"plain_n1e3", "dielectric_n1e4", "adjoint_n1e5"}
    for name, e in out.items():
        for kind in ("explicit_rbe", "full_k_sum"):
            assert e[kind]["ms_per_eval"] > 0 and e[kind]["particle_evals_per_s"] > 0, (name, kind)
            assert "scaled by" in e[kind]["sample"]
        assert e["full_k_sum"]["wave_vectors"] > e["P"]
