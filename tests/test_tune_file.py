"""The autotuner's tile-shape file (include/gfdeconv.h, gfdeconv_tune_read):
format, ranges and errors, read by the library on the host (no GPU)."""
import pytest

gfd = pytest.importorskip("paper_1609_01839_gb300")


def write(tmp_path, text):
    p = tmp_path / "tune.txt"
    p.write_text(text)
    return str(p)


def test_missing_file_is_an_empty_table(tmp_path):
    assert gfd.tune_read(str(tmp_path / "absent.txt")) == (4, {})


def test_reads_chains_and_classes(tmp_path):
    path = write(tmp_path, "# comment\nchains 2\n"
                           "class 1024 1024 col_threads 128 row_threads 256 gf_rows 32  # tail\n"
                           "\nclass 256 512 col_threads 64 row_threads 64 gf_rows 16\n")
    assert gfd.tune_read(path) == (2, {(1024, 1024): (128, 256, 32), (256, 512): (64, 64, 16)})


def test_later_line_for_the_same_canvas_wins(tmp_path):
    path = write(tmp_path, "class 512 512 col_threads 64 row_threads 64 gf_rows 16\n"
                           "class 512 512 col_threads 256 row_threads 128 gf_rows 64\n")
    assert gfd.tune_read(path) == (4, {(512, 512): (256, 128, 64)})


@pytest.mark.parametrize("text", [
    "chains 0\n",                                                      # not a chain count
    "chains 8\n",
    "class 1000 1024 col_threads 128 row_threads 256 gf_rows 32\n",    # canvas not 2^k
    "class 1024 1024 col_threads 512 row_threads 256 gf_rows 32\n",    # outside the search
    "class 1024 1024 col_threads 128 row_threads 256 gf_rows 8\n",
    "class 1024 1024 col_threads 128 row_threads 256\n",               # truncated
    "rows 4\n",                                                        # unknown keyword
])
def test_malformed_files_are_rejected(tmp_path, text):
    with pytest.raises(gfd.GfdError) as e:
        gfd.tune_read(write(tmp_path, text))
    assert e.value.code == -1
