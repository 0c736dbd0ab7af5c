"""Host logic of the serving loop that needs no GPU: cutting a large request
into pieces of whole columns."""
import numpy as np

from paper_2203_02293_b300.serve import Request, split_request


def test_split_request_covers_the_columns_in_order():
    r = Request(rid=7, arrival=0.5, n_cols=13, L=40, NB=30, cols=np.arange(100, 113), cube_base=1000, n_g=20)
    per_col = 30 * 20
    pieces = split_request(r, 4 * per_col + 5)          # room for 4 columns per piece
    assert [p.n_cols for p in pieces] == [4, 4, 4, 1]
    assert np.array_equal(np.concatenate([p.cols for p in pieces]), r.cols)
    assert [p.cube_base for p in pieces] == [1000 + j * 40 * per_col for j in (0, 4, 8, 12)]
    assert all(p.parent is r and p.rid == r.rid and p.arrival == r.arrival for p in pieces)
    assert r.pieces == pieces and r.pieces_left == 4
    assert sum(p.systems for p in pieces) == r.systems


def test_small_requests_and_single_columns_stay_whole():
    r = Request(rid=1, arrival=0.0, n_cols=3, L=10, NB=5, cols=np.arange(3), cube_base=0, n_g=20)
    assert split_request(r, 0) == [r] and split_request(r, r.systems) == [r]
    one = Request(rid=2, arrival=0.0, n_cols=1, L=10, NB=300, cols=np.arange(1), cube_base=0, n_g=20)
    assert split_request(one, 10) == [one]
    # a cap below one column still makes one-column pieces
    r = Request(rid=3, arrival=0.0, n_cols=3, L=10, NB=5, cols=np.arange(3), cube_base=0, n_g=20)
    assert [p.n_cols for p in split_request(r, 1)] == [1, 1, 1]
