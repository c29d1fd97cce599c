"""Pin of the oracle's sign convention for the factor columns (Algorithm 2 step 5 with
reading c5): each column of U^(n) is multiplied by -1 when its entry of largest magnitude
is negative; among entries of equal largest magnitude the one with the lowest row index
decides.  Every expected array below is written out by hand from that rule, not computed
by the function under test."""
import numpy as np

from oracle.rbki import sign_fix


def test_largest_entry_negative_flips_the_column():
    u = np.array([[0.1], [-0.9], [0.3]])
    np.testing.assert_array_equal(sign_fix(u), np.array([[-0.1], [0.9], [-0.3]]))


def test_largest_entry_positive_keeps_the_column():
    u = np.array([[-0.2], [0.05], [0.7], [-0.6]])
    np.testing.assert_array_equal(sign_fix(u), np.array([[-0.2], [0.05], [0.7], [-0.6]]))


def test_tie_of_equal_entries_lower_row_wins():
    # rows 1 and 3 tie at |0.6|; both negative: the column flips
    u = np.array([[0.2], [-0.6], [0.1], [-0.6]])
    np.testing.assert_array_equal(sign_fix(u), np.array([[-0.2], [0.6], [-0.1], [0.6]]))


def test_tie_of_opposite_signs_lower_row_decides():
    # rows 0 and 2 tie at |0.5|: row 0 is positive, so nothing changes ...
    u = np.array([[0.5], [0.3], [-0.5]])
    np.testing.assert_array_equal(sign_fix(u), np.array([[0.5], [0.3], [-0.5]]))
    # ... and with the signs swapped row 0 is negative, so the column flips
    v = np.array([[-0.5], [0.3], [0.5]])
    np.testing.assert_array_equal(sign_fix(v), np.array([[0.5], [-0.3], [-0.5]]))


def test_columns_are_fixed_independently_and_the_input_is_untouched():
    u = np.array([[0.6, -0.1, 0.0],
                  [-0.8, 0.2, -1.0],
                  [0.0, -0.3, 0.0]])
    expected = np.array([[-0.6, 0.1, -0.0],
                         [0.8, -0.2, 1.0],
                         [-0.0, 0.3, -0.0]])
    before = u.copy()
    out = sign_fix(u)
    np.testing.assert_array_equal(out, expected)
    np.testing.assert_array_equal(u, before)


def test_exact_zero_column_is_left_alone():
    u = np.array([[0.0, 1.0], [0.0, 0.0]])
    np.testing.assert_array_equal(sign_fix(u), np.array([[0.0, 1.0], [0.0, 0.0]]))
