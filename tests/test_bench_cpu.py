"""bench.py's reference arm on the CPU: the FP64 oracle timed on a bounded sample of the 128^3
workload, printed as one JSON line with the keys the benchmark contract names."""
import json


class _Args:
    steps = 1
    warmup = 0
    gpus = 1


def test_reference_arm_json_line(capsys):
    import bench
    bench.run_reference(_Args, 1, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "element-steps/s" and line["value"] > 0
    assert line["config"]["elements"] == 128 ** 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_algorithmic_bytes_per_element_step():
    """The roofline numerator: 144 B per hexahedron (28 FP32 conductances, 8 int32 ids) plus 28 B
    per node in the FP32 form."""
    import bench
    import fedfem_inputs as fi
    p = fi.nonlinear_cube(4, "hex")
    assert bench.algorithmic_bytes(p, 32) == 144 * p.n_elems + 28 * p.n_nodes
    assert bench.algorithmic_bytes(p, 64) == (28 * 8 + 8 * 4) * p.n_elems + 32 * p.n_nodes
