"""The batched path's work-granularity table (rbki_wave_tune_*): defaults, load / save round
trip, refusal of malformed files.  Host-side only: no GPU needed."""
import pytest

import paper_2211_14828_gb300 as rb
from paper_2211_14828_gb300 import _binding as B


@pytest.fixture(autouse=True)
def _reset():
    rb.rbki_wave_tune_reset()
    yield
    rb.rbki_wave_tune_reset()


def test_defaults():
    t = rb.rbki_wave_tune_table()
    assert t == {"gram": [16] * 8, "ttm": [4] * 8}


def test_load_save_round_trip(tmp_path):
    src = tmp_path / "tune.txt"
    src.write_text("# a table\ngram 0 2\ngram 7 64\nttm 3 8\n")
    rb.rbki_wave_tune_load(src)
    t = rb.rbki_wave_tune_table()
    assert t["gram"][0] == 2 and t["gram"][7] == 64 and t["ttm"][3] == 8
    assert t["gram"][1] == 16 and t["ttm"][0] == 4          # unlisted entries keep the defaults
    out = tmp_path / "saved.txt"
    rb.rbki_wave_tune_save(out)
    lines = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert len(lines) == 16 and "gram 7 64" in lines and "ttm 3 8" in lines
    rb.rbki_wave_tune_reset()
    rb.rbki_wave_tune_load(out)
    assert rb.rbki_wave_tune_table() == t


@pytest.mark.parametrize("text", ["gram 8 4\n", "gram 0 0\n", "ttm 1\n", "svd 0 4\n", "gram x 4\n"])
def test_malformed_file_is_refused(tmp_path, text):
    f = tmp_path / "bad.txt"
    f.write_text(text)
    with pytest.raises(rb.RbkiError) as e:
        rb.rbki_wave_tune_load(f)
    assert e.value.status == B.E_INVAL
    assert rb.rbki_wave_tune_table() == {"gram": [16] * 8, "ttm": [4] * 8}


def test_missing_file(tmp_path):
    with pytest.raises(rb.RbkiError) as e:
        rb.rbki_wave_tune_load(tmp_path / "none.txt")
    assert e.value.status == B.E_NOTFOUND
