"""Repository checks that need no GPU: the build compiles every CUDA source, and every profiling
command recorded under profiles/ leaves the GPU clocks alone and runs committed files only."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_build_lists_every_cuda_source():
    from paper_1205_6113_gb300 import build
    csrc = os.path.join(ROOT, "paper_1205_6113_gb300", "csrc")
    on_disk = sorted(f for f in os.listdir(csrc) if f.endswith(".cu"))
    assert sorted(build.SOURCES) == on_disk


def test_profile_commands_leave_clocks_alone():
    pdir = os.path.join(ROOT, "profiles")
    files = [f for f in os.listdir(pdir) if f.endswith(".md")]
    assert files
    for f in files:
        text = open(os.path.join(pdir, f)).read()
        blocks = re.findall(r"```\n(.*?)```", text, flags=re.S)
        cmds = [b for b in blocks if "ncu " in b]
        assert cmds, f
        for c in cmds:
            assert "--clock-control none" in c, f
            for script in re.findall(r"python ([\w/]+\.py)", c):
                assert os.path.exists(os.path.join(ROOT, script)), (f, script)
            assert "_work" not in c, f
