"""The mode-sum autotuner's cache file (BZ_TUNE_CACHE): a fresh process reads
the recorded choice instead of timing, and appends what it times."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROBE = ("import sys; sys.path.insert(0, %r); from paper_2103_14890_gb300 import binding as bz; "
         "m = bz.Modes(bz.Grid(2, 20, 10.0), 1.0); print(m.modesum_variant)" % ROOT)


def _run(cache):
    env = dict(os.environ, BZ_TUNE_CACHE=str(cache))
    env.pop("BZ_MODESUM_VARIANT", None)
    out = subprocess.run([sys.executable, "-c", PROBE], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    return int(out.stdout.split()[-1])


def test_cache_is_written_then_read(tmp_path):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cache = tmp_path / "tune.txt"
    cache.write_text("")
    v = _run(cache)                                   # times the variants, records the choice
    lines = [l.split() for l in cache.read_text().splitlines() if l.strip()]
    assert lines == [["2", "20", str(sms), str(v)]]
    # a recorded choice is used as is (here a different one than timed, if possible)
    other = 2 if v != 2 else 1
    cache.write_text("2 20 %d %d\n" % (sms, other))
    assert _run(cache) == other
    assert cache.read_text().count("\n") == 1         # nothing appended when the cache answered
