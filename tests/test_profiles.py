"""The ncu summaries under profiles/ name the command that produced them,
and that command runs committed files only (bench.py with its modes)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_profile_names_a_command_of_committed_files():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    for f in files:
        text = open(f).read()
        assert "ncu " in text and "--clock-control none" in text, f
        assert "_work/" not in text, f
        for script in re.findall(r"python ([\w./-]+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), (f, script)
