"""Host logic of bench.py that needs no GPU: the convergence counts that
decide whether a timed rate may be claimed, the provenance of the per-kernel
FP64 counts used by the roofline object, and the CPU description of the
baseline."""
import bench


def _step(newton, converged, gmres_ok):
    return {"newton_iterations": newton, "converged": converged, "gmres_converged": gmres_ok}


def test_convergence_counts_capped_steps_and_solves():
    stats = [_step(3, True, [1, 1, 1]), _step(20, False, [1] * 19 + [0]), _step(2, True, [0, 1])]
    c = bench.convergence(stats)
    assert c == {"steps_converged": 2, "steps_timed": 3, "newton_capped": 1, "gmres_capped": 2,
                 "linear_solves": 25}


def test_kernel_counts_match_the_profiled_sources():
    """The FP64 instruction and DRAM counts per cell in bench.py come from an
    ncu capture of the Jacobian-free kernels; their source hash must be that
    of the kernels as they are now, or the roofline object would report
    counts of other code (it flags them as stale at run time)."""
    assert bench.kernel_source_hash() == bench.KERNEL_COUNTS_HASH
    for table in (bench.FP64_INST_PER_CELL, bench.FP64_PIPE_INST_PER_CELL, bench.FP64_FLOPS_PER_CELL,
                  bench.INT_PIPE_OPS_PER_CELL, bench.DRAM_BYTES_PER_CELL_128, bench.HBM_BYTES_PER_CELL):
        assert set(table) == set(bench.JV_KERNELS)
    for k in bench.JV_KERNELS:
        assert bench.FP64_PIPE_INST_PER_CELL[k] >= bench.FP64_INST_PER_CELL[k]
        assert bench.FP64_FLOPS_PER_CELL[k] >= bench.FP64_INST_PER_CELL[k] + bench.INT_PIPE_OPS_PER_CELL[k]


def test_cpu_info_names_the_host():
    info = bench.cpu_info()
    assert info["logical_cores"] >= 1 and info["machine"]
