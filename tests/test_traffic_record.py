"""The committed ncu traffic record of the step kernel (profiles/step_kernel_traffic.md), which
bench.py reports as `roofline.traffic`, was taken on the current kernel source: its kernel_hash
matches the hash of lks_step.cu + lks_device.cuh (comments and spacing removed).  A change to the
kernel's code fails this test until the capture is repeated and the record updated."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_step_kernel_traffic_record_is_current():
    bench = _bench()
    traffic = bench._ncu_traffic("f32", 4096)
    assert traffic is not None, "profiles/step_kernel_traffic.md has no line for kernel_hash " + bench._kernel_hash()
    # one read of the source buffer plus most of the writes: between 0.8 and 1.0 of 152 B per node
    assert 0.8 * 152 * 4096 ** 2 < traffic <= 152 * 4096 ** 2


def test_comment_edits_do_not_change_the_hash():
    bench = _bench()
    code = "int f(int a) { return a + 1; }"
    assert bench._code_only("/* note */ " + code + " // more\n") == bench._code_only(code)
    assert bench._code_only(code.replace("+ 1", "+ 2")) != bench._code_only(code)
